/*
 * gs_b300.h -- C ABI of the B300 (sm_103a) 3D Gaussian Splatting training hot path.
 *
 * Method: GS-Scale (arXiv 2509.15645).  One training iteration (§2.4, steps 1-6)
 * is: frustum cull of every Gaussian -> gather of the visible subset (with the
 * deferred-update restore of §4.3.3 applied on the fly) -> differentiable tile
 * rasterizer (EWA projection, tile keys, key sort, front-to-back alpha
 * compositing, and its adjoint) -> deferred Adam (Eqs. 2-3, Fig. 10, §4.3.2).
 *
 * Conventions for every call
 *  - Pointers marked "device" point to CUDA device memory on the context's
 *    device; "host" pointers to ordinary host memory.  The caller owns every
 *    buffer it passes; the context owns only its scratch workspace and the
 *    pinned host buffers of its host-tier steps (allocated by gs_create).
 *  - Every call is asynchronous on the given stream (a cudaStream_t passed as
 *    void*; NULL = legacy default stream) and never synchronises, except
 *    gs_sync_status, gs_create/gs_destroy, gs_timing_read, gs_autotune,
 *    gs_split_point (once per bisection round) and gs_step on a host-tier scene
 *    (which waits once for its chunk-touch map, or, for GS_TIER_HOST_CPU_OPT,
 *    for its visible set and its update-set size).  A context
 *    must be driven from one stream at a time.
 *  - Invalid arguments return GS_ERR_INVALID_ARG before anything is launched;
 *    a failed launch returns GS_ERR_CUDA.  Errors found on the device (a
 *    capacity overflow, a non-finite loss) are latched in a device status word
 *    and returned by the next gs_sync_status.  Nothing traps or asserts.
 *  - Counts that depend on the data (the number of visible Gaussians, the
 *    number of tile keys) stay on the device; kernels read them there, so a
 *    whole step can be captured in a CUDA graph.
 *
 * Parameter layout (§2.3: 59 parameters per Gaussian at SH degree 3):
 * structure of arrays, plane r of Gaussian i at [r * pitch + i]:
 *   geo  rows 0..2 mean, 3..5 log-scale, 6..9 quaternion (w,x,y,z),
 *        10 opacity logit                                  (11 planes, fp32)
 *   sh   row 3k + c = SH coefficient k of colour c,  k < (L+1)^2
 *                                                    (3 (L+1)^2 planes)
 * D = 11 + 3 (L+1)^2 (14 at degree 0, 59 at degree 3).  Optimizer moments
 * m, v use the same D planes in the same order (geo planes first, then sh).
 * Compact per-visible-Gaussian arrays use planes of pitch `cap` (a capacity):
 * [r * cap + k] for the k-th visible Gaussian.
 */
#ifndef GS_B300_H
#define GS_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,
    GS_ERR_OOM = 2,
    GS_ERR_CUDA = 3,
    GS_ERR_BUDGET = 4,
    GS_ERR_CAPACITY = 5,   /* more visible Gaussians or tile keys than the context holds */
    GS_ERR_TIMEOUT = 6,
    GS_ERR_NUMERIC = 7     /* non-finite loss */
} gs_status;

/* Storage precision of SH planes and of the moments m, v.  The BF16 forms keep
 * the 11 geometry/opacity planes in fp32 (the "master" copy), store SH planes
 * and all moments in bf16, and compute everything in fp32.  GS_BF16_SH_MOM
 * rounds every bf16 store stochastically (deterministic counter-based hash of
 * seed, step, plane, index), which keeps small Adam updates and the 0.999
 * decay of v from being rounded away; GS_BF16_SH_MOM_RN rounds to nearest. */
enum { GS_FP32 = 0, GS_BF16_SH_MOM = 1, GS_BF16_SH_MOM_RN = 2 };

/* Residency of a scene's state (§4.2 selective offloading).  GS_TIER_DEVICE:
 * every plane in device memory.  GS_TIER_HOST_SH: the geometry and opacity
 * planes with their moments and restore directions stay in device memory
 * (geo, m, v, rdir then hold those 11 rows only, [11][pitch]); the SH planes
 * with their m and v live in pinned host memory (host_sh, host_m, host_v, each
 * [D-11][pitch] of the SH type; their restore directions are recomputed from
 * m, v on the device instead of being streamed).  gs_step streams the chunks
 * of 2^chunk_shift Gaussians that a step touches (the visible ones and the
 * optimizer's update set) into the context's staging ring with
 * cudaMemcpy2DAsync on one side stream and the updated rows back on another,
 * so both PCIe directions run at once; consecutive steps alternate between the
 * two halves of the ring when a step's chunks fit in one (a chunk the previous
 * step had visible is then copied between the halves on the device).  A step
 * synchronises the host once, for its chunk map, and waits for the previous
 * step's work if that ran on another stream.  The last write-backs of a step run
 * on past the end of its work on `stream` (overlapping the next step's cull);
 * gs_wait_copies makes a stream wait for them, gs_sync_status waits for them
 * on the host, and the next gs_step orders its own copies after them. */
/* GS_TIER_HOST_CPU_OPT: the paper's own offloaded configuration, with the
 * optimizer of the SH planes on the host cores (§4.2.2 parameter forwarding,
 * §4.3 deferred update with OpenMP), for comparison with GS_TIER_HOST_SH,
 * whose SH rows are stepped by device kernels.  The scene is laid out as in
 * GS_TIER_HOST_SH except that host_sh, host_m and host_v are Gaussian-major,
 * [pitch][D-11] (the row of Gaussian i at i * (D-11)), fp32 only; the context
 * needs gs_config.cpu_opt = 1.  Per
 * gs_step: the cull (with the optimizer's select) on the device and one host
 * synchronisation for the step's visible Gaussians (the union over its views)
 * and their defer counters; the host forwards their SH values (the previous
 * step's pending update applied to its members, the deferred restore of the
 * others; nothing is written to the host planes) into a pinned block that goes
 * to the device in pieces as they are ready; a worker thread then applies the
 * previous step's update to the host planes while the device renders,
 * back-propagates and steps the geometry planes; the step's SH gradients, its
 * update set and the delays come back into host buffers and are applied by
 * the next gs_step (or by gs_sync_status, which also waits for the worker).
 * Read host_sh, host_m, host_v only after gs_sync_status.  The step
 * synchronises the host twice (visible set; update-set size). */
enum { GS_TIER_DEVICE = 0, GS_TIER_HOST_SH = 1, GS_TIER_HOST_CPU_OPT = 2 };

/* Adam variants: deferred with the restore tables of Fig. 10 (the method) or
 * eager (Eq. 1 on every Gaussian each step: the baseline the paper improves). */
enum { GS_ADAM_DEFERRED = 0, GS_ADAM_EAGER = 2 };

typedef struct gs_ctx gs_ctx;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  R is the
 * world->camera rotation (row-major), t the translation: p_cam = R mu + t.
 * Pixel (i, j) has its centre at (i + 0.5, j + 0.5).
 *
 * Regions (image splitting, §4.4): with full_width = 0 (and x0 = y0 = 0) the
 * camera renders its whole width x height image.  Otherwise it renders the
 * region [x0, x0 + width) x [y0, y0 + height) of the full_width x full_height
 * image of the same camera (fx, fy, cx, cy are the full image's): pixel (i, j)
 * of the region is pixel (x0 + i, y0 + j) of the full image, the projection's
 * guard band is the full image's, and the L1 loss of the region is normalised
 * by the full image's 3 * full_width * full_height values, so the losses and
 * gradients of a view's regions, summed, are the whole view's.  The cull keeps
 * a Gaussian whose 3-sigma square overlaps the region's tiles; regions that
 * start on a tile boundary of the full image keep the full image's tile grid,
 * and the union of their visible sets is the whole view's. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float near_z, far_z;
    int32_t width, height;
    int32_t x0, y0;                   /* region origin in the full image */
    int32_t full_width, full_height;  /* 0: the camera is the whole image */
} gs_camera;

/* A Gaussian set with its optimizer state (device pointers, except host_*). */
typedef struct {
    int64_t n;             /* number of Gaussians (< 2^31) */
    int64_t pitch;         /* elements between planes, >= n, multiple of 4 */
    int32_t sh_degree;     /* 0..3 */
    int32_t precision;     /* GS_FP32, GS_BF16_SH_MOM or GS_BF16_SH_MOM_RN (sh, m, v stored as bf16) */
    float *geo;            /* [11][pitch] fp32 */
    void *sh;              /* [3 (L+1)^2][pitch] fp32 or bf16 (unused in GS_TIER_HOST_SH) */
    void *m;               /* [D][pitch] fp32 or bf16 ([11][pitch] in GS_TIER_HOST_SH), NULL = no optimizer
                              state (render only) */
    void *v;               /* like m */
    float *rdir;           /* restore direction m / (sqrt(v) + eps) of each geometry parameter, kept by the
                              optimizer so the cull's deferred restore of every Gaussian is one multiply-add:
                              [11][pitch] fp32 (a larger buffer is accepted; nothing past row 11 is read or
                              written: the SH planes' directions are taken from m and v by the few restores
                              that need them).  Must equal that expression (all zero when m = v = 0; see
                              gs_refresh_rdir).  NULL: the kernels recompute it from m and v */
    uint8_t *counter;      /* [n] defer counters of §4.3.2 (0..max_defer) */
    int32_t step;          /* optimizer steps completed; the next step is step + 1 */
    int32_t tier;          /* GS_TIER_DEVICE, GS_TIER_HOST_SH or GS_TIER_HOST_CPU_OPT */
    void *host_sh;         /* host tiers only: host [D-11][pitch] SH planes (pinned for GS_TIER_HOST_SH), */
    void *host_m;          /*   their first moments, */
    void *host_v;          /*   and second moments (all of the SH type) */
    void *host_rdir;       /*   unused (SH restore directions are recomputed from m, v on the device); may be NULL */
} gs_scene;

/* Optimizers of the deferred update (§4.3: Adam is the method's; the paper
 * names SGD with momentum and AdamW as optimizers the deferral carries over
 * to).  GS_OPT_ADAM: Eq. 1.  GS_OPT_ADAMW: decoupled weight decay (each step
 * w <- (1 - lr weight_decay) w, then the Adam step); its catch-up over d
 * deferred steps is w <- (1 - lr weight_decay)^d w - wlut[d] m / (sqrt(v) +
 * eps), Fig. 10's table with its i-th term weighted by (1 - lr
 * weight_decay)^(i-1).  GS_OPT_SGDM: SGD with momentum mu = beta1 (b <- mu b
 * + g, w <- w - lr b; no dampening; beta2 and eps unused; b lives in the m
 * planes, v is neither read nor written); its catch-up is exact: w <- w - lr
 * (mu + ... + mu^d) b, b <- mu^d b. */
enum { GS_OPT_ADAM = 0, GS_OPT_ADAMW = 1, GS_OPT_SGDM = 2 };

/* Optimizer hyper-parameters (§4.3.2).  lr per parameter group:
 * 0 mean, 1 log-scale, 2 quaternion, 3 opacity, 4 SH DC, 5 SH rest. */
typedef struct {
    float lr[6];
    float beta1, beta2, eps;
    int32_t max_defer;     /* MAX of the counter, at most 15 (4-bit counter) */
    int32_t mode;          /* GS_ADAM_DEFERRED or GS_ADAM_EAGER */
    int32_t seed;          /* stochastic-rounding seed of the BF16 form */
    int32_t optimizer;     /* GS_OPT_ADAM (0), GS_OPT_ADAMW or GS_OPT_SGDM */
    float weight_decay;    /* GS_OPT_ADAMW: decoupled decay lambda >= 0 with lr[g] * lambda < 1; else unused */
} gs_adam_cfg;

/* Context capacities, fixed at creation. */
typedef struct {
    int64_t max_gaussians;   /* largest scene n */
    int64_t max_visible;     /* capacity of the compact visible set per view */
    int64_t max_keys;        /* capacity of (tile, Gaussian) keys per view */
    int32_t max_width, max_height;
    int32_t tile_w, tile_h;  /* raster tile: tile_w in {4, 8, 16, 32, 64}, tile_w * tile_h in {32, 64, 128, 256} */
    int32_t max_views;       /* views per gs_step, 1..8 */
    int32_t max_sh_degree;   /* 0..3 */
    int64_t stage_chunks;    /* staging ring of host-tier scenes, in chunks (0: no host tier) */
    int32_t chunk_shift;     /* log2 Gaussians per chunk, 10..20 (0: 11) */
    int32_t stage_elem_bytes;/* element size of the staged SH rows: 4 (0: 4) serves every form, 2 only the bf16 forms */
    int32_t render_views;    /* views whose render buffers (splats, tile lists, images) exist at once, 1..max_views
                                (0: max_views).  gs_step renders its views in rounds of this many through the same
                                buffers, gradients summed over the rounds, so the working set is bounded by one
                                round (a view split into regions, §4.4, with render_views = 1 holds one region's
                                buffers at a time); the cull buffers (masks, ids) are kept for max_views views */
    int32_t list_records;    /* 1: also keep each view's splat records in list order (48 bytes per key of
                                capacity), which the TMA-staged rasterizer variant 9 needs; 0: variant 9 is not
                                available on this context */
    int32_t cpu_opt;         /* 1: the context can step GS_TIER_HOST_CPU_OPT scenes (device: a [D-11][per-step
                                visible capacity] fp32 block of forwarded SH rows and the visible ids and counters;
                                host: pinned buffers for the same block, two steps' SH gradients and update sets
                                of up to max_gaussians members); 0: it cannot */
} gs_config;

/* ------------------------------------------------------------------ context */

/* Bytes of device workspace a context with this configuration needs. */
GS_API gs_status gs_workspace_size(const gs_config *cfg, size_t *bytes);

/* Create a context on `device`.  `workspace` (device, >= gs_workspace_size
 * bytes, 256-byte aligned) is borrowed for the context's lifetime; pass NULL
 * to let the context allocate it itself.  *out receives the handle. */
GS_API gs_status gs_create(gs_ctx **out, const gs_config *cfg, int device, void *workspace, size_t workspace_bytes);

/* Release the context (and the workspace it allocated, if any). */
GS_API gs_status gs_destroy(gs_ctx *ctx);

/* Text of the last error recorded on this context (never NULL). */
GS_API const char *gs_last_error(const gs_ctx *ctx);

/* Synchronise `stream`, then return and clear the first error latched on the
 * device since the last call (GS_OK if none). */
GS_API gs_status gs_sync_status(gs_ctx *ctx, void *stream);

/* Make `stream` wait (without blocking the host) for the host-tier copies
 * the context has in flight: the write-backs of its last gs_step.  Work
 * enqueued on `stream` afterwards sees the updated host planes.  A no-op for
 * contexts without a staging ring. */
GS_API gs_status gs_wait_copies(gs_ctx *ctx, void *stream);

/* Device pointer to the context's 8 int32 counters: [0] visible count of the
 * last gs_cull, [1] key count of the last render, [2] update-set size of the
 * last deferred Adam step, [3] latched status, [6] Gaussians of the last
 * render whose 2D covariance went through the FP64 chain, [7] Gaussians that
 * passed the cull's conservative pre-test in the last gs_step (the cull reads
 * their rotation planes; the others leave after the mean and scale planes). */
GS_API const int32_t *gs_device_counters(const gs_ctx *ctx);

/* ------------------------------------------------------------------ hot path */

/* Frustum cull (§2.4 step 1; done on the GPU as in §4.2.1).  For every
 * Gaussian: 3D near/far test, EWA projection of its covariance, 3-sigma radius
 * and tile rectangle, and the 2D image-bounds test.  If `adam` is non-NULL and
 * the scene has optimizer state, the geometry is first restored with the
 * deferred-update tables of the coming step (§4.3.3), without modifying it.
 * Outputs (device): ids_out[max_visible] = visible Gaussian indices in
 * ascending order, *n_vis_out = their count (clamped to max_visible; overflow
 * latches GS_ERR_CAPACITY).  The visibility bitmask stays in the context for
 * the next gs_adam_deferred. */
GS_API gs_status gs_cull(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cam, const gs_adam_cfg *adam,
                  int32_t *ids_out, int32_t *n_vis_out, void *stream);

/* Render one view (§2.4 steps 1-3) of the Gaussians ids[0..*n_vis) (device,
 * ascending, from gs_cull): gather with restore (as gs_cull), projection and
 * SH colour, each tile's list of the splats that can reach it sorted by depth
 * (ties by Gaussian id), front-to-back compositing on a black background.
 * image_out (device fp32 [3][H][W]).  The context keeps what the
 * backward needs (compact parameters, splats, sorted keys, tile ranges) until
 * the next gs_render_fwd. */
GS_API gs_status gs_render_fwd(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cam, const gs_adam_cfg *adam,
                        const int32_t *ids, const int32_t *n_vis, float *image_out, void *stream);

/* Adjoint of the last gs_render_fwd (§2.4 step 5): dL_dimage (device fp32
 * [3][H][W]) -> grad_compact (device fp32 [D][cap], row r of the k-th visible
 * Gaussian at [r * cap + k]; cap >= that render's visible count), overwritten.
 * Transmittance is recomputed per tile, not stored per pixel. */
GS_API gs_status gs_render_bwd(gs_ctx *ctx, const float *dL_dimage, float *grad_compact, int64_t cap, void *stream);

/* L1 loss of §2.4 step 4: *loss_out = mean |image - target| over `count`
 * values; dL_dimage = sign(image - target) / count.  All device fp32. */
GS_API gs_status gs_loss_l1(gs_ctx *ctx, const float *image, const float *target, int64_t count, float *loss_out,
                     float *dL_dimage, void *stream);

/* One optimizer step (§4.3, Eqs. 1-3).  ids/n_vis (device) are the Gaussians
 * with a gradient this step (ascending; the last gs_cull's visibility mask in
 * the context must describe the same set), grad_compact (device fp32 [D][cap])
 * their gradients.  Deferred mode: update set = ids U {counter == max_defer};
 * each member is restored through the tables, stepped with Eq. 1 and its
 * counter cleared; every other counter is incremented.  Eager mode: every
 * Gaussian is stepped.  Increments scene->step. */
GS_API gs_status gs_adam_deferred(gs_ctx *ctx, gs_scene *scene, const int32_t *ids, const int32_t *n_vis,
                           const float *grad_compact, int64_t cap, const gs_adam_cfg *adam, void *stream);

/* Recompute scene->rdir = m / (sqrt(v) + eps) for every parameter (after m or
 * v were set by other means, or eps changed). */
GS_API gs_status gs_refresh_rdir(gs_ctx *ctx, const gs_scene *scene, const gs_adam_cfg *adam, void *stream);

/* The current (eager-equivalent) parameters and moments without modifying the
 * scene: catch-up of each Gaussian's deferred steps (tests, checkpoints).
 * Outputs (device fp32 [D][pitch], may be NULL). */
GS_API gs_status gs_adam_materialize(gs_ctx *ctx, const gs_scene *scene, const gs_adam_cfg *adam, float *w_out,
                              float *m_out, float *v_out, void *stream);

/* The tables the deferred update of optimizer step `step` (>= 1: the step a
 * scene with scene->step == step - 1 takes next) hands to the kernels, fp32,
 * computed in double from the hyper-parameters (Fig. 10, §4.3.2):
 *   param     [6][16] row-major: per parameter group g and delay d, the
 *             coefficient of the restore w <- decay[g][d] w - param[g][d] dir
 *             with dir = m / (sqrt(v) + eps) (Adam, AdamW) or the momentum
 *             buffer b (SGDM), i.e. the sum over the d skipped steps of Eq.
 *             3's weights; 0 for d = 0, d > max_defer and d >= step;
 *   mom, var  [16]: beta1^(d+1), beta2^(d+1), the decay of m and v over the
 *             d skipped steps and the current one (SGDM: mu^(d+1), and 1);
 *   step_size [6]: lr[g] / (1 - beta1^step) (SGDM: lr[g]);
 *   bias_corr: sqrt(1 - beta2^step) (SGDM: 1);
 *   decay     [6][16]: (1 - lr[g] weight_decay)^d for AdamW, else 1.
 * Host arrays owned by the caller; any may be NULL.  Touches no device.
 * GS_ERR_INVALID_ARG for a NULL adam, step < 1 or hyper-parameters the
 * optimizer cannot use (max_defer outside [1, 15], ...). */
GS_API gs_status gs_adam_tables(const gs_adam_cfg *adam, int32_t step, float *param, float *mom, float *var,
                                float *step_size, float *bias_corr, float *decay);

/* Scatter compact gradients to a full [D][pitch] array (zero elsewhere). */
GS_API gs_status gs_grad_scatter(gs_ctx *ctx, const gs_scene *scene, const int32_t *ids, const int32_t *n_vis,
                          const float *grad_compact, int64_t cap, float *grad_full, void *stream);

/* One whole training iteration on n_views views (§2.4 steps 1-6): cull every
 * view, render, L1 loss against targets[v] (device fp32 [3][H][W] each),
 * backward, gradients summed over the views, one optimizer step over the union
 * of the visible sets.  *loss_out (device) = sum over views of the L1 losses.
 * The views may be the regions of one split view (§4.4; targets[v] then holds
 * the region's pixels): the step is then the whole view's.  Replays a CUDA
 * graph captured on the first call with the same scene pointers, view count
 * and image sizes.  Increments scene->step. */
GS_API gs_status gs_step(gs_ctx *ctx, gs_scene *scene, const gs_camera *views, const float *const *targets,
                  int32_t n_views, const gs_adam_cfg *adam, float *loss_out, void *stream);

/* Stage timing of gs_step with CUDA events (benchmarks).  After
 * gs_timing_enable(ctx, max_steps), each gs_step records events on its stream
 * around: the whole step, the first view's cull kernel, its render forward and
 * backward, the optimizer stage, the optimizer's apply kernel (the D-plane
 * sweep) and the first view's rasterizer backward kernel.  gs_timing_read synchronises the device, writes elapsed
 * milliseconds ms_out[step * GS_TIMING_SPANS + span] for up to max_steps
 * recorded steps, stores their number in *steps_out and restarts recording.
 * Enabling or disabling timing re-captures the step graph. */
enum { GS_SPAN_STEP = 0, GS_SPAN_CULL = 1, GS_SPAN_FWD = 2, GS_SPAN_BWD = 3, GS_SPAN_ADAM = 4,
       GS_SPAN_ADAM_APPLY = 5, GS_SPAN_RASTER_BWD = 6, GS_TIMING_SPANS = 7 };
GS_API gs_status gs_timing_enable(gs_ctx *ctx, int32_t max_steps);
GS_API gs_status gs_timing_read(gs_ctx *ctx, float *ms_out, int32_t max_steps, int32_t *steps_out);

/* Rasterizer variants.  v < 6: one tile per block, pixels per thread
 * 1 << (v >> 1) and a shared-memory splat batch of (v & 1 ? 256 : 128)
 * records; a tile shape allows them when tile_h is a multiple of the pixels
 * per thread and the block has 32 to 256 threads.  v = 6, 7 (32-pixel tiles
 * only): one tile per warp, 4 warps per block with batches of 64 records, or
 * 8 warps with batches of 32.  v = 8 (32-pixel tiles only): as 7, walking the
 * list two entries at a time with paired FP32 (f32x2) arithmetic.  v = 9
 * (32-pixel tiles, contexts with list_records only): as 7, each batch staged
 * in shared memory by one TMA bulk copy of the tile's records, written in
 * list order by the first rasterizer pass that uses them (48 bytes per key
 * of extra traffic).  Every variant computes the same image bit
 * for bit; they differ only in speed. */
#define GS_RASTER_VARIANTS 10

/* Autotuner: time every variant the context's tile shape allows on this scene
 * and view (render forward and backward separately; CUDA events, best of
 * three) and keep the fastest forward and the fastest backward for this
 * context.  Synchronises the stream; call it outside stream capture.
 * chosen_out (host, 2 ints, may be NULL) receives the forward and the backward
 * variant, ms_out (host, 2 * GS_RASTER_VARIANTS floats, may be NULL) the
 * forward stage's milliseconds of each variant, then the backward stage's (-1
 * where not allowed).  gs_set_raster_variant sets both. */
GS_API gs_status gs_autotune(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cam, int32_t *chosen_out,
                             float *ms_out, void *stream);

/* Select a rasterizer variant explicitly (tests); GS_ERR_INVALID_ARG if the
 * tile shape does not allow it. */
GS_API gs_status gs_set_raster_variant(gs_ctx *ctx, int32_t variant);

/* Select the forward and the backward rasterizer variant separately (as the
 * autotuner does); GS_ERR_INVALID_ARG if the context does not allow either. */
GS_API gs_status gs_set_raster_variants(gs_ctx *ctx, int32_t fwd, int32_t bwd);

/* Work counts of the rasterizer backward for one view (benchmarks): renders
 * forward and backward once (the rendered image as dL/dimage) with a counting
 * instance of the backward kernel and writes counts[0] = (pixel, splat) pairs
 * that pass the 3-sigma square test, counts[1] = pairs that contribute
 * (alpha >= 1/255 before the transmittance stop) and counts[2] = (tile, splat)
 * keys of the lists that no pixel of their tile takes as a contributor
 * (32-pixel tiles; 0 for other tile shapes).  counts: host, 3 entries.
 * Synchronises the stream. */
GS_API gs_status gs_raster_pair_counts(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cam, uint64_t *counts,
                                       void *stream);

/* Densification on deferred optimizer state (§2.4 step 7 with §4.3; the
 * paper leaves the rules to 3DGS).  For Gaussian i of `src` (resident, with
 * optimizer state, after src->step steps): g = grad_accum[i] / denom[i] (0
 * where denom[i] <= 0), the mean view-space gradient norm the caller
 * accumulated; the current (caught-up) values decide: g >= grad_threshold
 * clones it when its largest scale is at most percent_dense * extent and
 * splits it into two children otherwise (children: scales / 1.6, means mu +
 * R(q) (s * z_j) with z_j = normals[(j * 3 + a) * n + i], a = 0..2, j = 0, 1,
 * standard normal values the caller draws); every Gaussian whose opacity
 * sigmoid(logit) is below min_opacity is dropped together with its copies.
 * A cloned row is caught up (its moments decayed over its deferred steps, its
 * counter 0) and its clone starts with zero moments; split rows are replaced
 * by their children (zero moments, counter 0); every other row keeps its
 * stored values, restore directions and counter.  `dst` (device arrays of the
 * same degree and precision, rdir present iff src has it, capacity
 * dst->pitch) receives the survivors in their order, then the clones, then
 * the first children, then the second children; dst->n and dst->step are set.
 * Synchronises the stream once (to read the counts).  GS_ERR_CAPACITY, with
 * dst->n set to the count needed and nothing written, if dst->pitch is too
 * small.  grad_accum, denom: device fp32 [n]; normals: device fp32 [2][3][n]. */
GS_API gs_status gs_densify(gs_ctx *ctx, const gs_scene *src, gs_scene *dst, const gs_adam_cfg *adam,
                            const float *grad_accum, const float *denom, const float *normals, float extent,
                            float grad_threshold, float percent_dense, float min_opacity, void *stream);

/* Number of kernel launches in the captured gs_step graph (0 before the first
 * gs_step). */
GS_API gs_status gs_step_kernel_count(const gs_ctx *ctx, int32_t *kernels);

/* Largest scene gs_cull_noalloc accepts. */
#define GS_CULL_NOALLOC_MAX_GAUSSIANS (1 << 24)

/* gs_cull without a context and without any device allocation.  The paper has
 * no counterpart: this exists for callers that cannot call cudaMalloc (and so
 * cannot create a gs_ctx with its own workspace), e.g. code inside a framework
 * whose memory pool owns all device memory, loops that forbid allocation after
 * start-up, or callers that must keep a fixed device footprint.  Same
 * arguments and results as gs_cull on a context with tile size tile_w x
 * tile_h: ids_out (device, room for scene->n ids) receives the visible
 * Gaussians in ascending order and *n_vis_out (device) their count.
 * status_out (device, may be NULL) receives the status the kernels found on
 * the device: GS_OK, or GS_ERR_TIMEOUT if a cull block gave up waiting for its
 * own copies (*n_vis_out is then 0).
 * Its scratch is a fixed ~2.1 MB array of device memory inside the library,
 * held on every GPU that loads the library until the process exits.
 * Returns GS_ERR_CAPACITY, launching nothing, if scene->n exceeds
 * GS_CULL_NOALLOC_MAX_GAUSSIANS, and GS_ERR_INVALID_ARG, launching nothing,
 * for the arguments gs_cull rejects (sh_degree outside 0..3, a non-finite or
 * non-positive focal length, unusable Adam hyper-parameters, ...).  The first
 * call on each device looks up that array's address (with the device current)
 * and should come before any stream capture.  All calls share the array, so
 * calls that overlap on the GPU race; serialise them (one stream, or events). */
GS_API gs_status gs_cull_noalloc(const gs_scene *scene, const gs_camera *cam, const gs_adam_cfg *adam, int32_t tile_w,
                                 int32_t tile_h, int32_t *ids_out, int32_t *n_vis_out, int32_t *status_out,
                                 void *stream);

/* Failure-path testing (no counterpart in the paper).  Every cull block (and
 * every warp of the TMA-staged rasterizer, variant 9) waits on an mbarrier
 * for the TMA copies it issued itself, each wait bounded; after `first_wait`
 * polls (default 2^24) of its first wait it gives up: latches GS_ERR_TIMEOUT
 * (gs_sync_status returns it), lets the copies it issued land (waiting for
 * them with the default bound) and returns, so the context stays usable.  0
 * makes every one give up at once.  ctx = NULL sets the limit of
 * gs_cull_noalloc (process-wide).  Host only; gs_step captures a new graph
 * after a change. */
GS_API gs_status gs_set_cull_wait_limit(gs_ctx *ctx, uint32_t first_wait);

/* Inspection of the last gs_render_fwd (tests, debugging).  Device pointers,
 * owned by the context, valid until the next render: *tile_of_key[K] and
 * *splat_of_key[K] the (tile id, compact visible index) pairs in sorted order,
 * *n_keys the count K, *ranges[2 * tiles] the [begin, end) of each tile. */
GS_API gs_status gs_render_lists(const gs_ctx *ctx, const uint32_t **tile_of_key, const uint32_t **splat_of_key,
                                 const int32_t **n_keys, const uint32_t **ranges);

/* Deferred optimizer step on host arrays, on the host cores (§4.3 with
 * OpenMP: the update GS_TIER_HOST_CPU_OPT applies to its SH planes, callable
 * alone).  w, m, v: host fp32, Gaussian-major: the value of parameter row
 * plane0 + r of Gaussian i at [i * row + r] (0 <= r < planes <= row,
 * plane0 + planes <= 59; learning-rate group of each row as in gs_step),
 * Gaussians 0 .. n_rows - 1.  uids[0..n_upd): the update set, ascending ids
 * below n_rows, with udelay its delays (0..max_defer); vids[0..n_vis):
 * ascending ids with a gradient row, grad[k * grow + r] the gradient of row
 * plane0 + r of Gaussian vids[k] (grow >= planes); members without a row step
 * with zero gradient.  One step t = step (>= 1) with the tables of
 * gs_adam_tables(adam, step), in FP32 (IEEE square root and division).
 * threads <= 0: every core.  Errors (nothing written): GS_ERR_INVALID_ARG for a
 * null array with a non-zero count, bad sizes, ids out of order or out of
 * range, or an invalid adam (mode must be deferred).  All memory is the
 * caller's. */
GS_API gs_status gs_cpu_deferred_step(float *w, float *m, float *v, int64_t n_rows, int32_t row, int32_t plane0,
                                      int32_t planes, const int32_t *uids, const uint8_t *udelay, int64_t n_upd,
                                      const int32_t *vids, const float *grad, int64_t n_vis, int64_t grow,
                                      const gs_adam_cfg *adam, int32_t step, int32_t threads);

/* Parameter forwarding (§4.2.2) on host arrays: out[r * opitch + k] (host,
 * plane-major, opitch >= n) = row plane0 + r of Gaussian ids[k] as the next
 * step, step + 1, sees it, without writing w, m, v (laid out as in
 * gs_cpu_deferred_step).  counter[k]: that Gaussian's defer counter at step + 1;
 * > 0 restores over counter[k] deferred steps (tables of step + 1), 0 applies
 * the pending update of step `step` (uids .. grow as in gs_cpu_deferred_step;
 * n_upd = 0 for none) if ids[k] is one of its members, else takes the stored
 * value.  ids ascending.  Errors as gs_cpu_deferred_step (step >= 0 here). */
GS_API gs_status gs_cpu_forward(const float *w, const float *m, const float *v, int64_t n_rows, int32_t row,
                                int32_t plane0, int32_t planes, const int32_t *ids, const uint8_t *counter, int64_t n,
                                const int32_t *uids, const uint8_t *udelay, int64_t n_upd, const int32_t *vids,
                                const float *grad, int64_t n_vis, int64_t grow, const gs_adam_cfg *adam,
                                int32_t step, float *out, int64_t opitch, int32_t threads);

/* OpenMP threads of the host-core optimizer of GS_TIER_HOST_CPU_OPT steps
 * (<= 0: every core; the default). */
GS_API gs_status gs_set_cpu_threads(gs_ctx *ctx, int32_t threads);

/* The last GS_TIER_HOST_CPU_OPT gs_step: stats[0] host ms forwarding the
 * visible rows, [1] host ms of the worker's update (the previous step's),
 * [2] host ms the step waited for that worker, [3] bytes host -> device,
 * [4] bytes device -> host, [5] rows forwarded, [6] members in the update
 * set the step left pending. */
GS_API gs_status gs_cpu_tier_stats(const gs_ctx *ctx, double *stats);

/* Host tier: chunks staged by the last gs_step of a GS_TIER_HOST_SH scene and
 * the bytes it moved between host and device (both directions). */
GS_API gs_status gs_host_tier_stats(const gs_ctx *ctx, int64_t *chunks, int64_t *bytes);

/* Balance-aware split point of one view (§4.4): the tile boundary along
 * `axis` (0: a vertical line, regions left | right; 1: a horizontal line,
 * regions top | bottom) that divides the view into two regions of about equal
 * visible-Gaussian counts.  Bisection over the tile boundaries 0 < s < tiles
 * (tiles along the axis): lo = 0, hi = tiles; each of `steps` rounds culls
 * both regions at s = clamp((lo + hi) / 2, 1, tiles - 1) in one sweep, then
 * sets hi = s if the first region has more visible Gaussians than the second
 * (the split moves into the fuller region, shrinking it), else lo = s.  The
 * result is s = clamp((lo + hi) / 2, 1, tiles - 1); the paper takes 5 rounds.
 * *split_out = the chosen boundary in pixels (a multiple of the tile size
 * along the axis); counts_out[0..1] (may be NULL) = the two regions' visible
 * counts at that split.  cam is a whole image (full_width = 0) with at least
 * two tiles along the axis.  Culls with the deferred restore when the scene has
 * optimizer state and adam is deferred, as gs_cull does.  Synchronises with
 * the stream once per round (the counts are read on the host); uses the
 * context's per-view cull buffers of views 0 and 1. */
GS_API gs_status gs_split_point(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cam, const gs_adam_cfg *adam,
                                int32_t axis, int32_t steps, int32_t *split_out, int64_t *counts_out, void *stream);

/* Inspection of the last gs_render_fwd: the projected splats of the visible
 * set in compact order (entry k belongs to ids[k]), device pointers owned by
 * the context and valid until the next render.  *geom[4 * k + 0..3] = (mean2d
 * x, mean2d y, pixel radius, opacity), *conic[4 * k + 0..3] = (inverse 2D
 * covariance entries A, B, C, camera depth) (§2.4 steps 1-2); *n_vis is the
 * device count.  Gaussians that were not kept have radius 0 or an empty tile
 * rectangle. */
GS_API gs_status gs_render_splats(const gs_ctx *ctx, const float **geom, const float **conic, const int32_t **n_vis);

/* Inspection of the last gs_step: the gradients its optimizer used -- the
 * loss's gradient summed over the step's views (§2.4 step 5) for every
 * Gaussian a view saw -- as device pointers owned by the context, valid until
 * the next call that renders or culls: (*grad)[r * (*pitch) + k] is the
 * gradient of parameter row r of Gaussian (*ids)[k], for k below the device
 * count **n, ids ascending.  GS_ERR_INVALID_ARG before the first gs_step. */
GS_API gs_status gs_step_gradients(const gs_ctx *ctx, const float **grad, int64_t *pitch, const int32_t **ids,
                                   const int32_t **n);

#ifdef __cplusplus
}
#endif

#endif /* GS_B300_H */
