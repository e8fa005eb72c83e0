// gs_runtime.cu -- context, workspace, argument blocks and the C ABI of
// include/gs_b300.h.  No kernel arithmetic lives here: every step of the hot
// path is a kernel in k_cull.cu, k_scan.cu, k_render.cu or k_adam.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <array>
#include <vector>

#include <chrono>
#include <thread>

#include "cpu_opt.hpp"
#include "gs_kernels.cuh"
#include "host_plan.hpp"

using namespace gs;

namespace {

enum { SLOT_CULL = 0, SLOT_RENDER = 1, SLOT_ADAM = 2, SLOT_STEP = 3, N_SLOTS = 4 };

struct GraphCache {
    cudaGraph_t graph = nullptr;   // kept alive: its node handles address the exec's nodes
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t args_node = nullptr;
    cudaKernelNodeParams args_params{};
    // what the captured graph baked in
    float *geo = nullptr;
    void *sh = nullptr, *m = nullptr, *v = nullptr;
    float *rdir = nullptr;
    uint8_t *counter = nullptr;
    int64_t n = 0, pitch = 0;
    int deg = -1, n_views = 0, mode = -1, prec = -1, opt = -1;
    int W[MAX_VIEWS] = {0}, H[MAX_VIEWS] = {0};
    float *loss = nullptr;
    bool timed = false;
    int variant = -1;
    uint32_t first_wait = 0;
    cudaGraphNode_t ev_node[TP_COUNT] = {nullptr};
    int kernels = 0;
};

// GS_TIER_HOST_CPU_OPT: the host side of the paper's CPU-optimizer
// configuration.  A step's update (its members and delays, its visible ids and
// their SH gradients) is held in the buffer set of the step's parity until the
// next step forwards from it and a worker thread applies it.
struct CpuUpdateBuf {
    int32_t *uids = nullptr, *vids = nullptr;      // pinned [max_gaussians], [gcap]
    uint8_t *udelay = nullptr;                     // pinned [max_gaussians]
    float *grad = nullptr;                         // pinned [SH planes][gcap]
    int64_t n_upd = 0, n_vis = 0;
    bool have_upd = false;                         // uids / udelay copied
    bool full = false;                             // an update not yet applied to the host planes
    int32_t step = 0;                              // the step it belongs to
    DevLut lut{};
    int opt = GS_OPT_ADAM;
    HostPlanes planes{};                           // the host planes it applies to
};

struct CpuTierState {
    int threads = 0;                               // <= 0: every core
    float *stage_d = nullptr;                      // device [SH planes][gcap] forwarded rows (workspace)
    uint8_t *cnt_d = nullptr;                      // device [gcap] counters of the visible ids
    float *stage_h = nullptr;                      // pinned [SH planes][gcap]
    uint8_t *cnt_h = nullptr;                      // pinned [gcap]
    int *counts_h = nullptr;                       // pinned [2]: visible count, update-set size
    CpuUpdateBuf buf[2];
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev_up = nullptr, ev_grad = nullptr, ev_down = nullptr;
    bool down_pending = false;
    std::thread worker;
    double lazy_ms = 0.0;                          // written by the worker
    double fwd_ms = 0.0, wait_ms = 0.0;
    int64_t h2d = 0, d2h = 0, rows = 0, left = 0;
};

}  // namespace

struct gs_ctx {
    int device = 0;
    int num_sms = 148;
    gs_config cfg{};
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    DevArgs *args = nullptr;     // [N_SLOTS]
    Counters *cnt = nullptr;
    int *nvis_view = nullptr;    // [MAX_VIEWS] visible counts of gs_step's views
    int *n_render = nullptr;     // visible count of the last gs_render_fwd
    int *n_tmp = nullptr;
    unsigned long long *stats = nullptr;   // counters of gs_raster_pair_counts
    int64_t nwords = 0, nchunks = 0;
    uint32_t *mask = nullptr, *wprefix = nullptr, *chunk = nullptr;
    uint32_t *umask = nullptr, *uchunk = nullptr;
    int32_t *uids = nullptr;
    uint8_t *udelay = nullptr;
    uint32_t *amask = nullptr, *aprefix = nullptr, *achunk = nullptr;
    PairBufs pairs{};                   // the pair-wise optimizer apply
    uint32_t *vmask[MAX_VIEWS] = {nullptr};
    uint32_t *vchunk[MAX_VIEWS] = {nullptr};
    uint32_t *vprefix[MAX_VIEWS] = {nullptr};
    int32_t *vids[MAX_VIEWS] = {nullptr};
    uint32_t *union_mask = nullptr, *union_prefix = nullptr, *union_chunk = nullptr;
    int32_t *union_ids = nullptr;       // [gcap_u] ascending ids of the union of a step's views
    int last_views = 0;                 // views of the last gs_step (0: none yet)
    int64_t last_gpitch = 0;            // row pitch of its gradients in grad_u
    float *imgs[MAX_VIEWS] = {nullptr}, *dimgs[MAX_VIEWS] = {nullptr}, *grad_u = nullptr;
    int *work = nullptr;                // rasterizer work counters
    int64_t gcap_u = 0;
    RenderBufs rbs[MAX_VIEWS]{};
    Work w{};
    // state kept from the last gs_render_fwd for gs_render_bwd
    bool have_fwd = false;
    SceneView fwd_sc{};
    DevCam fwd_cam{};
    GraphCache graph;
    // stage timing
    int t_max = 0, t_used = 0;
    cudaEvent_t *t_events = nullptr;   // [t_max][TP_COUNT]
    // host tier: staging ring of SH rows (w, m, v, restore direction), each
    // [max SH planes][stage_chunks << shift], chunk -> slot tables, the copy
    // stream and its events
    int shift = 15;
    int64_t max_chunks = 0;
    void *stage[3] = {nullptr, nullptr, nullptr};
    int32_t *dslot = nullptr;
    uint8_t *dtouch = nullptr;
    uint8_t *htouch = nullptr;          // pinned
    int32_t *hslot = nullptr;           // pinned
    cudaStream_t cstream = nullptr;     // host -> device copies
    cudaStream_t dstream = nullptr;     // device -> host copies (the other PCIe direction, concurrently)
    cudaEvent_t ev_vis = nullptr, ev_upd = nullptr, ev_done = nullptr, ev_end = nullptr;
    cudaEvent_t ev_down[2] = {nullptr, nullptr};
    HostPlan plan;                      // the last host-tier step's slots, rounds and copy runs
    HostHistory hist;                   // what that step leaves for the next (ring halves)
    const void *pscene = nullptr;
    int64_t pn = 0;
    cudaEvent_t ev_half[2] = {nullptr, nullptr};   // write-backs of the last step that used half 0 / 1 done
    cudaEvent_t ev_sdone = nullptr;     // the previous host-tier step's work on its stream done
    int64_t last_touched = 0, last_bytes = 0;
    CpuTierState cpu;                   // GS_TIER_HOST_CPU_OPT (cfg.cpu_opt)
    char err[512] = {0};
};

static void timing_free(gs_ctx *c)
{
    if (c->t_events) {
        for (int k = 0; k < c->t_max * TP_COUNT; k++) cudaEventDestroy(c->t_events[k]);
        free(c->t_events);
    }
    c->t_events = nullptr;
    c->t_max = c->t_used = 0;
}

static gs_status fail(gs_ctx *c, gs_status st, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

static gs_status cuda_check(gs_ctx *c, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, GS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    return GS_OK;
}

static int n_params(int deg) { return N_GEO + 3 * (deg + 1) * (deg + 1); }

// ---------------------------------------------------------------------------
// Workspace layout.  The same walk sizes the workspace (base == nullptr) and
// hands out the pointers.
struct Carver {
    char *base;
    size_t off = 0;
    template <class T> T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static bool valid_cfg(const gs_config *c)
{
    if (!c) return false;
    int tp = c->tile_w * c->tile_h;
    return c->max_gaussians > 0 && c->max_gaussians < (1ll << 31) - CHUNK && c->max_visible > 0 &&
           c->max_visible < (1ll << 31) && c->max_keys > 0 && c->max_keys < (1ll << 32) - 1 && c->max_width > 0 &&
           c->max_height > 0 && c->tile_w >= 4 && c->tile_h > 0 && 64 % c->tile_w == 0 &&
           (tp == 32 || tp == 64 || tp == 128 || tp == 256) &&
           c->max_views >= 1 && c->max_views <= MAX_VIEWS && c->max_sh_degree >= 0 && c->max_sh_degree <= 3 &&
           c->max_width < 65536 * c->tile_w && c->max_height < 65536 * c->tile_h && c->stage_chunks >= 0 &&
           (c->chunk_shift == 0 || (c->chunk_shift >= 10 && c->chunk_shift <= 20)) &&
           (c->stage_elem_bytes == 0 || c->stage_elem_bytes == 2 || c->stage_elem_bytes == 4) &&
           c->render_views >= 0 && c->render_views <= c->max_views && (c->list_records == 0 || c->list_records == 1) &&
           (c->cpu_opt == 0 || c->cpu_opt == 1);
}

static int stage_eb(const gs_config &g) { return g.stage_elem_bytes ? g.stage_elem_bytes : 4; }

// Views rendered at once by gs_step (sets of render buffers).
static int render_slots(const gs_config &g) { return g.render_views ? g.render_views : g.max_views; }

static void carve(gs_ctx *c, char *base)
{
    const gs_config &g = c->cfg;
    Carver k{base};
    const int64_t N = g.max_gaussians, V = g.max_visible, K = g.max_keys;
    const int D = n_params(g.max_sh_degree);
    const int64_t NW = (N + 31) / 32 + CHUNK_WORDS, NC = (N + CHUNK - 1) / CHUNK + 1;
    const int64_t tiles = (int64_t)((g.max_width + g.tile_w - 1) / g.tile_w) * ((g.max_height + g.tile_h - 1) / g.tile_h);
    const int64_t P = 3ll * g.max_width * g.max_height;
    c->nwords = NW;
    c->nchunks = NC;
    c->args = k.take<DevArgs>(N_SLOTS);
    c->cnt = k.take<Counters>(1);
    c->nvis_view = k.take<int>(MAX_VIEWS);
    c->n_render = k.take<int>(1);
    c->n_tmp = k.take<int>(4);
    c->stats = k.take<unsigned long long>(4);
    c->mask = k.take<uint32_t>(NW);
    c->wprefix = k.take<uint32_t>(NW);
    c->chunk = k.take<uint32_t>(NC);
    c->umask = k.take<uint32_t>(NW);
    c->uchunk = k.take<uint32_t>(NC);
    c->uids = k.take<int32_t>(N);
    c->udelay = k.take<uint8_t>(N);
    c->pairs.pmask = k.take<uint32_t>(NW / 2 + CHUNK_WORDS);
    c->pairs.pchunk = k.take<uint32_t>(NC / 2 + 2);
    c->pairs.pids = k.take<int32_t>(N / 2 + 1);
    c->pairs.pinfo = k.take<uint32_t>(N / 2 + 1);
    c->pairs.n_pairs = k.take<int>(1);
    c->amask = k.take<uint32_t>(NW);
    c->aprefix = k.take<uint32_t>(NW);
    c->achunk = k.take<uint32_t>(NC);
    for (int v = 0; v < g.max_views; v++) {
        c->vmask[v] = k.take<uint32_t>(NW);
        c->vchunk[v] = k.take<uint32_t>(NC);
        c->vprefix[v] = k.take<uint32_t>(NW);
        c->vids[v] = k.take<int32_t>(V);
    }
    if (g.max_views > 1) {
        c->union_mask = k.take<uint32_t>(NW);
        c->union_prefix = k.take<uint32_t>(NW);
        c->union_chunk = k.take<uint32_t>(NC);
    }
    // render buffers of each view a step renders at once (a round)
    for (int v = 0; v < render_slots(g); v++) {
        RenderBufs &rb = c->rbs[v];
        rb.cap = V;
        rb.kcap = K;
        rb.compact = k.take<float>((size_t)D * V);
        rb.rec0 = k.take<float4>(V);
        rb.rec1 = k.take<float4>(V);
        rb.rec2 = k.take<float4>(V);
        rb.rect = k.take<uint2>(V);
        rb.depth = k.take<uint32_t>(V);
        rb.tile_cnt = k.take<uint32_t>(tiles + 1);
        rb.tile_cur = k.take<uint32_t>(tiles);
        rb.long_tiles = k.take<int32_t>(tiles);
        rb.first_tiles = k.take<int32_t>(tiles);
        for (int j = 0; j < 2; j++) {
            rb.tk[j] = k.take<uint32_t>(K);
            rb.tv[j] = k.take<uint32_t>(K);
        }
        rb.ranges = k.take<uint2>(tiles);
        rb.g9 = k.take<float>(G9_STRIDE * V);
        int *ctr = k.take<int>(2);
        rb.n_keys = v == 0 ? (base ? &c->cnt->n_keys : nullptr) : ctr;
        rb.n_fix = v == 0 ? (base ? &c->cnt->n_fix : nullptr) : ctr + 1;
        rb.cfinal = k.take<float>(P);
        rb.fix_idx = k.take<int32_t>(V);
        rb.fix_flag = k.take<uint8_t>(V);
        rb.n_big = k.take<int>(3);
        rb.big_idx = k.take<int32_t>(V);
        rb.reach = k.take<uint32_t>(V);
        rb.lrec = g.list_records ? k.take<float4>(3 * (size_t)K) : nullptr;
        c->imgs[v] = k.take<float>(P);
        c->dimgs[v] = k.take<float>(P);
    }
    c->work = k.take<int>(4);
    c->w.partials = k.take<uint32_t>(2048);
    c->gcap_u = g.max_views > 1 ? (N < (int64_t)g.max_views * V ? N : (int64_t)g.max_views * V) : V;
    c->grad_u = k.take<float>((size_t)D * c->gcap_u);
    if (g.max_views > 1) c->union_ids = k.take<int32_t>(c->gcap_u);
    if (g.cpu_opt) {
        c->cpu.stage_d = k.take<float>((size_t)(D - N_GEO) * c->gcap_u);
        c->cpu.cnt_d = k.take<uint8_t>(c->gcap_u);
    }
    if (g.stage_chunks > 0) {
        c->shift = g.chunk_shift ? g.chunk_shift : 11;
        c->max_chunks = (N + (1ll << c->shift) - 1) >> c->shift;
        const size_t ring = (size_t)(D - N_GEO) * ((size_t)g.stage_chunks << c->shift) * stage_eb(g);
        for (int j = 0; j < 3; j++) c->stage[j] = k.take<char>(ring);    // w, m, v
        c->dslot = k.take<int32_t>(c->max_chunks);
        c->dtouch = k.take<uint8_t>(c->max_chunks);
    }
    c->ws_bytes = k.off + 256;
}

// ---------------------------------------------------------------------------
// A region camera (§4.4 image splitting) renders part of the full image: its
// principal point moves by the region's origin, while the guard band and the
// loss normalisation stay the full image's.
bool gs::camera_region_ok(const gs_camera &a)
{
    if (a.full_width == 0) return a.x0 == 0 && a.y0 == 0 && a.full_height == 0;
    return a.full_width > 0 && a.full_height > 0 && a.x0 >= 0 && a.y0 >= 0 &&
           (int64_t)a.x0 + a.width <= a.full_width && (int64_t)a.y0 + a.height <= a.full_height;
}

DevCam gs::make_cam(const gs_camera &a, int tile_w, int tile_h)
{
    DevCam c{};
    const bool region = a.full_width > 0;
    const int FW = region ? a.full_width : a.width, FH = region ? a.full_height : a.height;
    memcpy(c.R, a.R, sizeof(c.R));
    memcpy(c.t, a.t, sizeof(c.t));
    c.fx = a.fx; c.fy = a.fy;
    c.cx = region ? (float)((double)a.cx - a.x0) : a.cx;
    c.cy = region ? (float)((double)a.cy - a.y0) : a.cy;
    c.near_z = a.near_z; c.far_z = a.far_z;
    c.limx = (float)(1.3 * (0.5 * FW / (double)a.fx));
    c.limy = (float)(1.3 * (0.5 * FH / (double)a.fy));
    c.loss_inv = 1.f / (float)(3 * (int64_t)FW * FH);
    for (int i = 0; i < 3; i++)
        c.campos[i] = (float)(-((double)a.R[0 * 3 + i] * a.t[0] + (double)a.R[1 * 3 + i] * a.t[1] + (double)a.R[2 * 3 + i] * a.t[2]));
    c.width = a.width;
    c.height = a.height;
    c.tile_w = tile_w;
    c.tile_h = tile_h;
    c.tiles_x = (a.width + tile_w - 1) / tile_w;
    c.tiles_y = (a.height + tile_h - 1) / tile_h;
    return c;
}

// Tables of the deferred update (Fig. 10, §4.3.2) for step t, computed in
// double and rounded to float.  Entries with delay >= t are never used.
// Adam: Fig. 10.  AdamW: the same recursion with its i-th term weighted by
// rho^(i-1), rho = 1 - lr wd, and the restore's decay rho^d.  Momentum SGD
// (mu = beta1): param[d] = lr (mu + ... + mu^d), the buffer decays by mu^(d+1)
// and takes the gradient with weight 1; no bias correction.
DevLut gs::make_lut(const gs_adam_cfg *a, int t, bool restore, int precision)
{
    DevLut L{};
    L.restore = 0;
    for (int g = 0; g < N_GROUPS; g++) {
        L.wdf[g] = 1.f;
        for (int i = 0; i < LUT_N; i++) L.decay[g][i] = 1.f;
    }
    if (!a) return L;
    L.seed = (uint32_t)a->seed;
    L.stochastic = precision == GS_BF16_SH_MOM ? 1 : 0;
    const int opt = a->optimizer;
    const double b1 = a->beta1, b2 = a->beta2;
    if (opt == GS_OPT_SGDM) {
        const double mu = b1;
        for (int g = 0; g < N_GROUPS; g++) {
            double acc = 0.0;
            L.param[g][0] = 0.f;
            for (int i = 1; i < LUT_N; i++) {
                acc = mu * acc + a->lr[g] * mu;
                L.param[g][i] = (i <= a->max_defer && i <= t - 1) ? (float)acc : 0.f;
            }
            L.step_size[g] = a->lr[g];
        }
        for (int i = 0; i < LUT_N; i++) {
            L.mom[i] = (float)std::pow(mu, i + 1);
            L.var[i] = 1.f;
        }
        L.bias_corr = L.inv_bias_corr = 1.f;
        L.omb1 = 1.f;
        L.omb2 = 0.f;
    } else {
        const double scale = b1 / std::sqrt(b2);
        for (int g = 0; g < N_GROUPS; g++) {
            const double rho = opt == GS_OPT_ADAMW ? 1.0 - (double)a->lr[g] * a->weight_decay : 1.0;
            double prev = 0.0;
            L.param[g][0] = 0.f;
            for (int i = 1; i < LUT_N; i++) {
                if (i <= a->max_defer && i <= t - 1) {
                    prev = scale * prev + std::pow(rho, i - 1) * (a->lr[g] * b1) /
                                              (std::sqrt(b2 / (1.0 - std::pow(b2, t - i))) * (1.0 - std::pow(b1, t - i)));
                    L.param[g][i] = (float)prev;
                } else {
                    L.param[g][i] = 0.f;
                }
                L.decay[g][i] = (float)std::pow(rho, i);
            }
            L.wdf[g] = (float)rho;
            L.step_size[g] = (float)(a->lr[g] / (1.0 - std::pow(b1, t)));
        }
        for (int i = 0; i < LUT_N; i++) {
            L.mom[i] = (float)std::pow(b1, i + 1);
            L.var[i] = (float)std::pow(b2, i + 1);
        }
        L.bias_corr = (float)std::sqrt(1.0 - std::pow(b2, t));
        L.inv_bias_corr = (float)(1.0 / std::sqrt(1.0 - std::pow(b2, t)));
        L.omb1 = (float)(1.0 - b1);
        L.omb2 = (float)(1.0 - b2);
    }
    L.eps = a->eps;
    L.b1 = a->beta1;
    L.b2 = a->beta2;
    L.max_defer = a->max_defer;
    L.step = t;
    L.restore = restore ? 1 : 0;
    return L;
}

__global__ void k_set_args(DevArgs a, DevArgs *dst)
{
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&a);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (int k = threadIdx.x; k < (int)(sizeof(DevArgs) / 4); k += blockDim.x) d[k] = src[k];
}

static void set_args(gs_ctx *c, int slot, const DevArgs &a, cudaStream_t s)
{
    k_set_args<<<1, 128, 0, s>>>(a, c->args + slot);
}

static bool valid_cam(const gs_ctx *c, const gs_camera *cam)
{
    return cam && cam->width > 0 && cam->height > 0 && cam->width <= c->cfg.max_width &&
           cam->height <= c->cfg.max_height && cam->fx > 0.f && cam->fy > 0.f && cam->far_z > cam->near_z &&
           std::isfinite(cam->fx) && std::isfinite(cam->fy) && camera_region_ok(*cam);
}

static int elem_bytes(int prec) { return prec == GS_FP32 ? 4 : 2; }

// Host-tier scenes are accepted only where `host_ok` (gs_cull, which reads the
// device-resident geometry, and gs_step, which stages the SH rows).
static gs_status scene_view(gs_ctx *c, const gs_scene *s, bool need_opt, SceneView &sv, bool host_ok = false)
{
    if (!s) return fail(c, GS_ERR_INVALID_ARG, "scene is NULL");
    if (s->n <= 0 || s->n > c->cfg.max_gaussians) return fail(c, GS_ERR_INVALID_ARG, "scene n=%lld out of range", (long long)s->n);
    if (s->pitch < s->n || (s->pitch & 3)) return fail(c, GS_ERR_INVALID_ARG, "pitch must be >= n and a multiple of 4");
    if (s->sh_degree < 0 || s->sh_degree > c->cfg.max_sh_degree) return fail(c, GS_ERR_INVALID_ARG, "sh_degree out of range");
    if (s->precision != GS_FP32 && s->precision != GS_BF16_SH_MOM && s->precision != GS_BF16_SH_MOM_RN)
        return fail(c, GS_ERR_INVALID_ARG, "unknown precision form");
    if (s->tier != GS_TIER_DEVICE && s->tier != GS_TIER_HOST_SH && s->tier != GS_TIER_HOST_CPU_OPT)
        return fail(c, GS_ERR_INVALID_ARG, "unknown tier");
    const bool cpu = s->tier == GS_TIER_HOST_CPU_OPT;
    const bool host = s->tier == GS_TIER_HOST_SH || cpu;
    if (host && !host_ok) return fail(c, GS_ERR_INVALID_ARG, "host-tier scenes run through gs_step (and gs_cull)");
    if (host && (!s->host_sh || !s->host_m || !s->host_v || !s->m || !s->v || !s->counter))
        return fail(c, GS_ERR_INVALID_ARG, "host tiers need host_sh/m/v planes and the geometry's optimizer state");
    if (host && !cpu && c->cfg.stage_chunks <= 0)
        return fail(c, GS_ERR_INVALID_ARG, "host tier needs a staging ring (stage_chunks)");
    if (cpu && (!c->cfg.cpu_opt || s->precision != GS_FP32))
        return fail(c, GS_ERR_INVALID_ARG, "GS_TIER_HOST_CPU_OPT needs a context with cpu_opt and an fp32 scene");
    if (host && !cpu && elem_bytes(s->precision) > stage_eb(c->cfg))
        return fail(c, GS_ERR_INVALID_ARG, "staging ring holds %d-byte rows, the scene's SH rows have %d bytes",
                    stage_eb(c->cfg), (int)elem_bytes(s->precision));
    if (!s->geo || (!host && !s->sh)) return fail(c, GS_ERR_INVALID_ARG, "geo/sh planes are NULL");
    if (need_opt && (!s->m || !s->v || !s->counter)) return fail(c, GS_ERR_INVALID_ARG, "optimizer state is NULL");
    const int64_t eb = elem_bytes(s->precision), P = s->pitch;
    sv.geo = s->geo;
    sv.m = s->m;
    sv.v = s->v;
    sv.rdir = (s->m && s->v) ? s->rdir : nullptr;
    sv.prec = s->precision;
    sv.tier = s->tier;
    sv.counter = s->counter;
    sv.n = s->n;
    sv.pitch = P;
    sv.deg = s->sh_degree;
    sv.D = n_params(s->sh_degree);
    sv.opt = GS_OPT_ADAM;      // callers with optimizer hyper-parameters set their kind
    if (!host) {
        sv.sh.w = s->sh;
        sv.sh.m = s->m ? (char *)s->m + N_GEO * P * eb : nullptr;
        sv.sh.v = s->v ? (char *)s->v + N_GEO * P * eb : nullptr;
        sv.sh.rdir = nullptr;       // SH directions are not kept: restores take them from m, v
        sv.sh.ppitch = P;
        sv.sh.slot = nullptr;
        sv.sh.shift = 0;
        sv.sh.cmask = sv.sh.cprefix = nullptr;
        sv.sh.current = 0;
    } else if (cpu) {
        // the step's forwarded SH rows, placed by the step (visibility mask and prefix)
        sv.sh = ShRows{};
        sv.sh.w = c->cpu.stage_d;
        sv.sh.ppitch = c->gcap_u;
        sv.sh.current = 1;
    } else {
        sv.sh.cmask = sv.sh.cprefix = nullptr;
        sv.sh.current = 0;
        // SH restore directions are not streamed: the kernels recompute them from the staged m, v
        sv.sh.w = c->stage[0];
        sv.sh.m = c->stage[1];
        sv.sh.v = c->stage[2];
        sv.sh.rdir = nullptr;
        sv.sh.ppitch = c->cfg.stage_chunks << c->shift;
        sv.sh.slot = c->dslot;
        sv.sh.shift = c->shift;
    }
    return GS_OK;
}

bool gs::valid_adam(const gs_adam_cfg *a)
{
    if (!a) return false;
    if (!(a->beta1 >= 0.f && a->beta1 < 1.f && a->beta2 >= 0.f && a->beta2 < 1.f && a->eps >= 0.f)) return false;
    if (a->max_defer < 1 || a->max_defer > LUT_N - 1) return false;
    if (a->optimizer != GS_OPT_ADAM && a->optimizer != GS_OPT_ADAMW && a->optimizer != GS_OPT_SGDM) return false;
    for (int g = 0; g < N_GROUPS; g++)
        if (!std::isfinite(a->lr[g])) return false;
    if (a->optimizer == GS_OPT_ADAMW) {
        if (!(a->weight_decay >= 0.f) || !std::isfinite(a->weight_decay)) return false;
        for (int g = 0; g < N_GROUPS; g++)
            if (!((double)a->lr[g] * a->weight_decay < 1.0)) return false;
    }
    return a->mode == GS_ADAM_DEFERRED || a->mode == GS_ADAM_EAGER;
}

// ---------------------------------------------------------------------------
extern "C" {

static gs_status cpu_flush(gs_ctx *c);

gs_status gs_workspace_size(const gs_config *cfg, size_t *bytes)
{
    if (!valid_cfg(cfg) || !bytes) return GS_ERR_INVALID_ARG;
    gs_ctx tmp;
    tmp.cfg = *cfg;
    carve(&tmp, nullptr);
    *bytes = tmp.ws_bytes;
    return GS_OK;
}

gs_status gs_create(gs_ctx **out, const gs_config *cfg, int device, void *workspace, size_t workspace_bytes)
{
    if (!out || !valid_cfg(cfg)) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    gs_ctx *c = new (std::nothrow) gs_ctx();
    if (!c) return GS_ERR_OOM;
    c->cfg = *cfg;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return GS_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    carve(c, nullptr);
    if (workspace) {
        if (workspace_bytes < c->ws_bytes || ((uintptr_t)workspace & 255)) {
            delete c;
            return GS_ERR_INVALID_ARG;
        }
        c->ws = workspace;
    } else {
        if (cudaMalloc(&c->ws, c->ws_bytes) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return GS_ERR_OOM;
        }
        c->own_ws = true;
    }
    carve(c, (char *)c->ws);
    c->w.status = &c->cnt->status;
    c->w.num_sms = c->num_sms;
    c->rbs[0].variant = 1;
    if (!raster_variant_ok(c->rbs[0].variant, cfg->tile_w, cfg->tile_h, cfg->list_records)) c->rbs[0].variant = 0;
    c->rbs[0].variant_bwd = c->rbs[0].variant;
    c->w.scan_grid = c->num_sms * 2 > 1024 ? 1024 : c->num_sms * 2;
    if (cudaMemset(c->cnt, 0, sizeof(Counters)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->w.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->w.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->w.ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        gs_destroy(c);
        return GS_ERR_CUDA;
    }
    if (cfg->stage_chunks > 0) {
        if (cudaHostAlloc((void **)&c->htouch, c->max_chunks, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&c->hslot, c->max_chunks * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c->dstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_vis, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_upd, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_end, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_down[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_down[1], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_half[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_half[1], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_sdone, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            gs_destroy(c);
            return GS_ERR_CUDA;
        }
    }
    if (cfg->cpu_opt) {
        CpuTierState &T = c->cpu;
        const int64_t planes = n_params(cfg->max_sh_degree) - N_GEO, G = c->gcap_u, N = cfg->max_gaussians;
        bool ok = cudaHostAlloc((void **)&T.stage_h, planes * G * sizeof(float), cudaHostAllocDefault) == cudaSuccess &&
                  cudaHostAlloc((void **)&T.cnt_h, G, cudaHostAllocDefault) == cudaSuccess &&
                  cudaHostAlloc((void **)&T.counts_h, 2 * sizeof(int), cudaHostAllocDefault) == cudaSuccess;
        for (int j = 0; j < 2 && ok; j++) {
            CpuUpdateBuf &B = T.buf[j];
            ok = cudaHostAlloc((void **)&B.uids, N * sizeof(int32_t), cudaHostAllocDefault) == cudaSuccess &&
                 cudaHostAlloc((void **)&B.udelay, N, cudaHostAllocDefault) == cudaSuccess &&
                 cudaHostAlloc((void **)&B.vids, G * sizeof(int32_t), cudaHostAllocDefault) == cudaSuccess &&
                 cudaHostAlloc((void **)&B.grad, planes * G * sizeof(float), cudaHostAllocDefault) == cudaSuccess;
        }
        ok = ok && cudaStreamCreateWithFlags(&T.up, cudaStreamNonBlocking) == cudaSuccess &&
             cudaStreamCreateWithFlags(&T.down, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&T.ev_up, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&T.ev_grad, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&T.ev_down, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            gs_destroy(c);
            return GS_ERR_OOM;
        }
    }
    *out = c;
    return GS_OK;
}

gs_status gs_destroy(gs_ctx *c)
{
    if (!c) return GS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    {
        CpuTierState &T = c->cpu;
        if (T.worker.joinable()) T.worker.join();
        if (T.up) cudaStreamSynchronize(T.up);
        if (T.down) cudaStreamSynchronize(T.down);
        for (cudaEvent_t e : {T.ev_up, T.ev_grad, T.ev_down})
            if (e) cudaEventDestroy(e);
        if (T.up) cudaStreamDestroy(T.up);
        if (T.down) cudaStreamDestroy(T.down);
        for (void *p : {(void *)T.stage_h, (void *)T.cnt_h, (void *)T.counts_h})
            if (p) cudaFreeHost(p);
        for (CpuUpdateBuf &B : T.buf)
            for (void *p : {(void *)B.uids, (void *)B.udelay, (void *)B.vids, (void *)B.grad})
                if (p) cudaFreeHost(p);
    }
    if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
    if (c->graph.graph) cudaGraphDestroy(c->graph.graph);
    timing_free(c);
    if (c->cstream) cudaStreamSynchronize(c->cstream);
    if (c->dstream) cudaStreamSynchronize(c->dstream);
    if (c->w.side) {
        cudaStreamSynchronize(c->w.side);
        cudaStreamDestroy(c->w.side);
    }
    for (cudaEvent_t e : {c->w.ev_fork, c->w.ev_join})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {c->ev_vis, c->ev_upd, c->ev_done, c->ev_end, c->ev_down[0], c->ev_down[1], c->ev_half[0],
                          c->ev_half[1], c->ev_sdone})
        if (e) cudaEventDestroy(e);
    if (c->cstream) cudaStreamDestroy(c->cstream);
    if (c->dstream) cudaStreamDestroy(c->dstream);
    if (c->htouch) cudaFreeHost(c->htouch);
    if (c->hslot) cudaFreeHost(c->hslot);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    delete c;
    return GS_OK;
}

const char *gs_last_error(const gs_ctx *c) { return c ? c->err : "null context"; }

const int32_t *gs_device_counters(const gs_ctx *c) { return c ? reinterpret_cast<const int32_t *>(c->cnt) : nullptr; }

gs_status gs_wait_copies(gs_ctx *c, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!c->dstream) return GS_OK;
    if (cudaStreamWaitEvent((cudaStream_t)stream, c->ev_end, 0) != cudaSuccess) return cuda_check(c, "gs_wait_copies");
    return GS_OK;
}

gs_status gs_sync_status(gs_ctx *c, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "gs_sync_status");
    if (c->cfg.cpu_opt) {               // host planes of GS_TIER_HOST_CPU_OPT scenes brought up to date
        const gs_status st = cpu_flush(c);
        if (st) return st;
    }
    if (c->cstream && cudaStreamSynchronize(c->cstream) != cudaSuccess) return cuda_check(c, "gs_sync_status copies");
    if (c->dstream && cudaStreamSynchronize(c->dstream) != cudaSuccess) return cuda_check(c, "gs_sync_status copies");
    int st = 0;
    if (cudaMemcpy(&st, &c->cnt->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_check(c, "gs_sync_status read");
    int zero = 0;
    cudaMemcpy(&c->cnt->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (st) fail(c, (gs_status)st, "device latched status %d", st);
    return (gs_status)st;
}

gs_status gs_cull(gs_ctx *c, const gs_scene *scene, const gs_camera *cam, const gs_adam_cfg *adam, int32_t *ids_out,
                  int32_t *n_vis_out, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, false, sv, true);
    if (st) return st;
    if (!valid_cam(c, cam)) return fail(c, GS_ERR_INVALID_ARG, "invalid camera");
    if (!ids_out || !n_vis_out) return fail(c, GS_ERR_INVALID_ARG, "NULL output");
    if (adam && !valid_adam(adam)) return fail(c, GS_ERR_INVALID_ARG, "invalid adam config");
    if (adam) sv.opt = adam->optimizer;
    cudaStream_t s = (cudaStream_t)stream;
    DevArgs a{};
    a.cam[0] = make_cam(*cam, c->cfg.tile_w, c->cfg.tile_h);
    a.lut = make_lut(adam, scene->step + 1, adam && adam->mode == GS_ADAM_DEFERRED && sv.m && sv.v && sv.counter);
    a.n_views = 1;
    set_args(c, SLOT_CULL, a, s);
    launch_cull(sv, c->args + SLOT_CULL, 0, c->mask, c->chunk, c->w, s);
    compact_mask(c->mask, sv.n, c->chunk, true, ids_out, c->wprefix, (int)c->cfg.max_visible, &c->cnt->n_vis, c->w, s);
    cudaMemcpyAsync(n_vis_out, &c->cnt->n_vis, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    return cuda_check(c, "gs_cull");
}

gs_status gs_split_point(gs_ctx *c, const gs_scene *scene, const gs_camera *cam, const gs_adam_cfg *adam,
                         int32_t axis, int32_t steps, int32_t *split_out, int64_t *counts_out, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, false, sv, true);
    if (st) return st;
    if (!valid_cam(c, cam) || cam->full_width != 0) return fail(c, GS_ERR_INVALID_ARG, "invalid camera (a whole image)");
    if (axis != 0 && axis != 1) return fail(c, GS_ERR_INVALID_ARG, "axis must be 0 (x) or 1 (y)");
    if (steps < 0 || steps > 32 || !split_out) return fail(c, GS_ERR_INVALID_ARG, "steps out of range or NULL output");
    if (adam && !valid_adam(adam)) return fail(c, GS_ERR_INVALID_ARG, "invalid adam config");
    if (adam) sv.opt = adam->optimizer;
    if (c->cfg.max_views < 2) return fail(c, GS_ERR_INVALID_ARG, "splitting needs a context with max_views >= 2");
    const int T = axis == 0 ? c->cfg.tile_w : c->cfg.tile_h;
    const int tiles = ((axis == 0 ? cam->width : cam->height) + T - 1) / T;
    if (tiles < 2) return fail(c, GS_ERR_INVALID_ARG, "fewer than two tiles along the split axis");
    cudaStream_t s = (cudaStream_t)stream;
    const bool restore = adam && adam->mode == GS_ADAM_DEFERRED && sv.m && sv.v && sv.counter;
    const int64_t nchunks = ((sv.n + 31) / 32 + CHUNK_WORDS - 1) / CHUNK_WORDS;
    int32_t cnt[2] = {0, 0};
    // visible counts of the two regions split at tile boundary `at`: one cull
    // sweep over both, exact totals of the per-chunk counts (no capacity)
    auto count = [&](int at) -> gs_status {
        gs_camera r[2] = {*cam, *cam};
        for (int v = 0; v < 2; v++) {
            r[v].full_width = cam->width;
            r[v].full_height = cam->height;
        }
        if (axis == 0) {
            r[0].width = at * T;
            r[1].x0 = at * T;
            r[1].width = cam->width - at * T;
        } else {
            r[0].height = at * T;
            r[1].y0 = at * T;
            r[1].height = cam->height - at * T;
        }
        DevArgs a{};
        for (int v = 0; v < 2; v++) a.cam[v] = make_cam(r[v], c->cfg.tile_w, c->cfg.tile_h);
        a.lut = make_lut(adam, scene->step + 1, restore);
        a.n_views = 2;
        set_args(c, SLOT_CULL, a, s);
        launch_cull_views(sv, c->args + SLOT_CULL, 2, c->vmask, c->vchunk, c->w, s);
        for (int v = 0; v < 2; v++) scan_counts(c->vchunk[v], nchunks, c->nvis_view + v, 0, c->w, s);
        cudaMemcpyAsync(cnt, c->nvis_view, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "gs_split_point");
        int dev_st = 0;
        if (cudaMemcpy(&dev_st, &c->cnt->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return cuda_check(c, "gs_split_point status");
        if (dev_st) return fail(c, (gs_status)dev_st, "device latched status %d during the split search", dev_st);
        return GS_OK;
    };
    auto inner = [&](int x) { return x < 1 ? 1 : (x > tiles - 1 ? tiles - 1 : x); };
    int lo = 0, hi = tiles;
    for (int k = 0; k < steps; k++) {
        const int at = inner((lo + hi) / 2);
        if ((st = count(at)) != GS_OK) return st;
        if (cnt[0] > cnt[1]) hi = at;
        else lo = at;
    }
    const int at = inner((lo + hi) / 2);
    if (counts_out) {
        if ((st = count(at)) != GS_OK) return st;
        counts_out[0] = cnt[0];
        counts_out[1] = cnt[1];
    }
    *split_out = at * T;
    return cuda_check(c, "gs_split_point");
}

gs_status gs_render_fwd(gs_ctx *c, const gs_scene *scene, const gs_camera *cam, const gs_adam_cfg *adam,
                        const int32_t *ids, const int32_t *n_vis, float *image_out, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, false, sv);
    if (st) return st;
    if (!valid_cam(c, cam)) return fail(c, GS_ERR_INVALID_ARG, "invalid camera");
    if (!ids || !n_vis || !image_out) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    if (adam && !valid_adam(adam)) return fail(c, GS_ERR_INVALID_ARG, "invalid adam config");
    if (adam) sv.opt = adam->optimizer;
    cudaStream_t s = (cudaStream_t)stream;
    DevArgs a{};
    a.cam[0] = make_cam(*cam, c->cfg.tile_w, c->cfg.tile_h);
    a.lut = make_lut(adam, scene->step + 1, adam && adam->mode == GS_ADAM_DEFERRED && sv.m && sv.v && sv.counter);
    a.n_views = 1;
    set_args(c, SLOT_RENDER, a, s);
    cudaMemcpyAsync(c->n_render, n_vis, sizeof(int), cudaMemcpyDeviceToDevice, s);
    render_forward(sv, c->args + SLOT_RENDER, 0, ids, c->n_render, c->rbs[0], a.cam[0], image_out, false, nullptr,
                   nullptr, c->w, s, c->work);
    c->have_fwd = true;
    c->fwd_sc = sv;
    c->fwd_cam = a.cam[0];
    return cuda_check(c, "gs_render_fwd");
}

gs_status gs_render_bwd(gs_ctx *c, const float *dL_dimage, float *grad_compact, int64_t cap, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!c->have_fwd) return fail(c, GS_ERR_INVALID_ARG, "gs_render_bwd without a gs_render_fwd");
    if (!dL_dimage || !grad_compact || cap <= 0) return fail(c, GS_ERR_INVALID_ARG, "invalid argument");
    cudaStream_t s = (cudaStream_t)stream;
    render_backward(c->fwd_sc, c->args + SLOT_RENDER, 0, c->n_render, c->rbs[0], c->fwd_cam, dL_dimage, grad_compact, cap,
                    nullptr, nullptr, nullptr, c->w, s, c->work);
    return cuda_check(c, "gs_render_bwd");
}

gs_status gs_loss_l1(gs_ctx *c, const float *image, const float *target, int64_t count, float *loss_out,
                     float *dL_dimage, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!image || !target || !loss_out || count <= 0) return fail(c, GS_ERR_INVALID_ARG, "invalid argument");
    launch_loss_l1(image, target, count, loss_out, dL_dimage, c->w, (cudaStream_t)stream);
    return cuda_check(c, "gs_loss_l1");
}

gs_status gs_adam_deferred(gs_ctx *c, gs_scene *scene, const int32_t *ids, const int32_t *n_vis,
                           const float *grad_compact, int64_t cap, const gs_adam_cfg *adam, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, true, sv);
    if (st) return st;
    if (!valid_adam(adam)) return fail(c, GS_ERR_INVALID_ARG, "invalid adam config");
    sv.opt = adam->optimizer;
    if (!ids || !n_vis || !grad_compact || cap <= 0) return fail(c, GS_ERR_INVALID_ARG, "invalid argument");
    cudaStream_t s = (cudaStream_t)stream;
    DevArgs a{};
    a.lut = make_lut(adam, scene->step + 1, adam->mode == GS_ADAM_DEFERRED, scene->precision);
    a.n_views = 0;
    set_args(c, SLOT_ADAM, a, s);
    int icap = (int)(cap < c->cfg.max_visible ? cap : c->cfg.max_visible);
    launch_ids_to_mask(ids, n_vis, icap, c->amask, sv.n, c->w, s);
    compact_mask(c->amask, sv.n, c->achunk, false, nullptr, c->aprefix, (int)sv.n, c->n_tmp, c->w, s);
    if (adam->mode == GS_ADAM_DEFERRED)
        launch_adam_deferred(sv, c->args + SLOT_ADAM, c->amask, c->aprefix, grad_compact, cap, c->umask, c->uchunk,
                             c->uids, c->udelay, &c->cnt->n_upd, c->w, s, &c->pairs);
    else
        launch_adam_eager(sv, c->args + SLOT_ADAM, c->amask, c->aprefix, grad_compact, cap, c->w, s);
    st = cuda_check(c, "gs_adam_deferred");
    if (!st) scene->step += 1;
    return st;
}

gs_status gs_adam_materialize(gs_ctx *c, const gs_scene *scene, const gs_adam_cfg *adam, float *w_out, float *m_out,
                              float *v_out, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, true, sv);
    if (st) return st;
    if (!valid_adam(adam)) return fail(c, GS_ERR_INVALID_ARG, "invalid adam config");
    sv.opt = adam->optimizer;
    cudaStream_t s = (cudaStream_t)stream;
    DevArgs a{};
    a.lut = make_lut(adam, scene->step + 1, true);
    set_args(c, SLOT_ADAM, a, s);
    launch_materialize(sv, c->args + SLOT_ADAM, w_out, m_out, v_out, c->w, s);
    return cuda_check(c, "gs_adam_materialize");
}

gs_status gs_refresh_rdir(gs_ctx *c, const gs_scene *scene, const gs_adam_cfg *adam, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, true, sv);
    if (st) return st;
    if (!valid_adam(adam)) return fail(c, GS_ERR_INVALID_ARG, "invalid adam config");
    sv.opt = adam->optimizer;
    if (!sv.rdir) return fail(c, GS_ERR_INVALID_ARG, "scene has no rdir planes");
    cudaStream_t s = (cudaStream_t)stream;
    DevArgs a{};
    a.lut = make_lut(adam, scene->step + 1, true);
    set_args(c, SLOT_ADAM, a, s);
    launch_refresh_rdir(sv, c->args + SLOT_ADAM, c->w, s);
    return cuda_check(c, "gs_refresh_rdir");
}

gs_status gs_grad_scatter(gs_ctx *c, const gs_scene *scene, const int32_t *ids, const int32_t *n_vis,
                          const float *grad_compact, int64_t cap, float *grad_full, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, false, sv);
    if (st) return st;
    if (!ids || !n_vis || !grad_compact || !grad_full || cap <= 0) return fail(c, GS_ERR_INVALID_ARG, "invalid argument");
    int icap = (int)(cap < c->cfg.max_visible ? cap : c->cfg.max_visible);
    launch_grad_scatter(ids, n_vis, icap, grad_compact, cap, sv.D, grad_full, sv.pitch, c->w, (cudaStream_t)stream);
    return cuda_check(c, "gs_grad_scatter");
}

gs_status gs_timing_enable(gs_ctx *c, int32_t max_steps)
{
    if (!c || max_steps < 0 || max_steps > 1000000) return GS_ERR_INVALID_ARG;
    // the cached step graph records into the events freed here: drop it (once
    // no replay is in flight) so the next gs_step captures a graph for the new
    // events, or none
    if (c->graph.exec && cudaDeviceSynchronize() != cudaSuccess) return cuda_check(c, "gs_timing_enable");
    if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
    if (c->graph.graph) cudaGraphDestroy(c->graph.graph);
    c->graph.exec = nullptr;
    c->graph.graph = nullptr;
    timing_free(c);
    if (max_steps == 0) return GS_OK;
    c->t_events = (cudaEvent_t *)calloc((size_t)max_steps * TP_COUNT, sizeof(cudaEvent_t));
    if (!c->t_events) return GS_ERR_OOM;
    c->t_max = max_steps;
    for (int k = 0; k < max_steps * TP_COUNT; k++)
        if (cudaEventCreate(&c->t_events[k]) != cudaSuccess) {
            c->t_max = k / TP_COUNT;
            timing_free(c);
            return cuda_check(c, "gs_timing_enable");
        }
    return GS_OK;
}

gs_status gs_timing_read(gs_ctx *c, float *ms_out, int32_t max_steps, int32_t *steps_out)
{
    if (!c || !ms_out || !steps_out) return GS_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_check(c, "gs_timing_read");
    static const int span[GS_TIMING_SPANS][2] = {{TP_STEP0, TP_STEP1}, {TP_CULL0, TP_CULL1}, {TP_FWD0, TP_FWD1},
                                                 {TP_BWD0, TP_BWD1}, {TP_ADAM0, TP_ADAM1}, {TP_APPLY0, TP_APPLY1},
                                                 {TP_RBWD0, TP_RBWD1}};
    int n = c->t_used < max_steps ? c->t_used : max_steps;
    for (int st = 0; st < n; st++) {
        cudaEvent_t *ev = c->t_events + (size_t)st * TP_COUNT;
        for (int k = 0; k < GS_TIMING_SPANS; k++) {
            float ms = -1.f;
            if (cudaEventElapsedTime(&ms, ev[span[k][0]], ev[span[k][1]]) != cudaSuccess) {
                cudaGetLastError();
                ms = -1.f;
            }
            ms_out[st * GS_TIMING_SPANS + k] = ms;
        }
    }
    *steps_out = n;
    c->t_used = 0;
    return GS_OK;
}

gs_status gs_set_raster_variants(gs_ctx *c, int32_t fwd, int32_t bwd)
{
    if (!c || !raster_variant_ok(fwd, c->cfg.tile_w, c->cfg.tile_h, c->cfg.list_records) ||
        !raster_variant_ok(bwd, c->cfg.tile_w, c->cfg.tile_h, c->cfg.list_records))
        return GS_ERR_INVALID_ARG;
    for (int v = 0; v < MAX_VIEWS; v++) {
        c->rbs[v].variant = fwd;
        c->rbs[v].variant_bwd = bwd;
    }
    return GS_OK;
}

gs_status gs_set_raster_variant(gs_ctx *c, int32_t variant)
{
    if (!c || !raster_variant_ok(variant, c->cfg.tile_w, c->cfg.tile_h, c->cfg.list_records))
        return GS_ERR_INVALID_ARG;
    c->rbs[0].variant = c->rbs[0].variant_bwd = variant;
    return GS_OK;
}

gs_status gs_autotune(gs_ctx *c, const gs_scene *scene, const gs_camera *cam, int32_t *chosen_out, float *ms_out,
                      void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, false, sv);
    if (st) return st;
    if (!valid_cam(c, cam)) return fail(c, GS_ERR_INVALID_ARG, "invalid camera");
    cudaStream_t s = (cudaStream_t)stream;
    DevArgs a{};
    a.cam[0] = make_cam(*cam, c->cfg.tile_w, c->cfg.tile_h);
    a.n_views = 1;
    set_args(c, SLOT_RENDER, a, s);
    int32_t *ids = c->vids[0];
    launch_cull(sv, c->args + SLOT_RENDER, 0, c->mask, c->chunk, c->w, s);
    compact_mask(c->mask, sv.n, c->chunk, true, ids, c->wprefix, (int)c->cfg.max_visible, c->n_render, c->w, s);
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    const int keep = c->rbs[0].variant, keep_b = c->rbs[0].variant_bwd;
    float best_f = 1e30f, best_b = 1e30f;
    int best_vf = keep, best_vb = keep_b;
    gs_status res = GS_OK;
    for (int v = 0; v < N_RASTER_VARIANTS && res == GS_OK; v++) {
        if (ms_out) ms_out[v] = ms_out[N_RASTER_VARIANTS + v] = -1.f;
        if (!raster_variant_ok(v, c->cfg.tile_w, c->cfg.tile_h, c->cfg.list_records)) continue;
        c->rbs[0].variant = c->rbs[0].variant_bwd = v;
        float fbest = 1e30f, bbest = 1e30f;
        for (int rep = 0; rep < 4; rep++) {
            cudaEventRecord(e0, s);
            render_forward(sv, c->args + SLOT_RENDER, 0, ids, c->n_render, c->rbs[0], a.cam[0], c->imgs[0], false, nullptr,
                           nullptr, c->w, s, c->work);
            cudaEventRecord(e1, s);
            // the rendered image itself serves as a dense dL/dimage; the TMA-staged
            // backward is timed as after another forward variant, writing its
            // list-order records itself
            if (v == RASTER_TMA_VARIANT) c->rbs[0].variant = 0;
            render_backward(sv, c->args + SLOT_RENDER, 0, c->n_render, c->rbs[0], a.cam[0], c->imgs[0], c->grad_u,
                            c->cfg.max_visible, nullptr, nullptr, nullptr, c->w, s, c->work);
            c->rbs[0].variant = v;
            cudaEventRecord(e2, s);
            if (cudaEventSynchronize(e2) != cudaSuccess) {
                res = cuda_check(c, "gs_autotune");
                break;
            }
            float fms = 0.f, bms = 0.f;
            cudaEventElapsedTime(&fms, e0, e1);
            cudaEventElapsedTime(&bms, e1, e2);
            if (rep > 0) {                                 // the first run warms caches and clocks
                fbest = fminf(fbest, fms);
                bbest = fminf(bbest, bms);
            }
        }
        if (res != GS_OK) break;
        if (ms_out) {
            ms_out[v] = fbest;
            ms_out[N_RASTER_VARIANTS + v] = bbest;
        }
        if (fbest < best_f) { best_f = fbest; best_vf = v; }
        if (bbest < best_b) { best_b = bbest; best_vb = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (res != GS_OK) {
        c->rbs[0].variant = keep;
        c->rbs[0].variant_bwd = keep_b;
        return res;
    }
    for (int v = 0; v < MAX_VIEWS; v++) {
        c->rbs[v].variant = best_vf;
        c->rbs[v].variant_bwd = best_vb;
    }
    c->have_fwd = false;
    if (chosen_out) {
        chosen_out[0] = best_vf;
        chosen_out[1] = best_vb;
    }
    return cuda_check(c, "gs_autotune");
}

gs_status gs_raster_pair_counts(gs_ctx *c, const gs_scene *scene, const gs_camera *cam, uint64_t *counts,
                                void *stream)
{
    if (!c || !counts) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, false, sv);
    if (st) return st;
    if (!valid_cam(c, cam)) return fail(c, GS_ERR_INVALID_ARG, "invalid camera");
    cudaStream_t s = (cudaStream_t)stream;
    DevArgs a{};
    a.cam[0] = make_cam(*cam, c->cfg.tile_w, c->cfg.tile_h);
    a.n_views = 1;
    set_args(c, SLOT_RENDER, a, s);
    int32_t *ids = c->vids[0];
    launch_cull(sv, c->args + SLOT_RENDER, 0, c->mask, c->chunk, c->w, s);
    compact_mask(c->mask, sv.n, c->chunk, true, ids, c->wprefix, (int)c->cfg.max_visible, c->n_render, c->w, s);
    unsigned long long *dev = c->stats;
    cudaMemsetAsync(dev, 0, 3 * sizeof(unsigned long long), s);
    render_forward(sv, c->args + SLOT_RENDER, 0, ids, c->n_render, c->rbs[0], a.cam[0], c->imgs[0], false, nullptr, nullptr,
                   c->w, s, c->work);
    // the empty-key count needs a warp-tile backward (one tile per warp): 7 where the tile shape allows it
    const int vb = c->rbs[0].variant_bwd;
    if (raster_variant_ok(7, c->cfg.tile_w, c->cfg.tile_h, false)) c->rbs[0].variant_bwd = 7;
    render_backward(sv, c->args + SLOT_RENDER, 0, c->n_render, c->rbs[0], a.cam[0], c->imgs[0], c->grad_u, c->cfg.max_visible,
                    nullptr, nullptr, nullptr, c->w, s, c->work, dev);
    c->rbs[0].variant_bwd = vb;
    unsigned long long host[3] = {0, 0, 0};
    if (cudaMemcpyAsync(host, dev, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_check(c, "gs_raster_pair_counts");
    for (int i = 0; i < 3; i++) counts[i] = host[i];
    c->have_fwd = false;
    return GS_OK;
}

gs_status gs_adam_tables(const gs_adam_cfg *adam, int32_t step, float *param, float *mom, float *var,
                         float *step_size, float *bias_corr, float *decay)
{
    if (!adam || step < 1 || !valid_adam(adam)) return GS_ERR_INVALID_ARG;
    const DevLut L = make_lut(adam, step, true);
    for (int g = 0; g < N_GROUPS; g++) {
        for (int i = 0; i < LUT_N; i++) {
            if (param) param[g * LUT_N + i] = L.param[g][i];
            if (decay) decay[g * LUT_N + i] = L.decay[g][i];
        }
        if (step_size) step_size[g] = L.step_size[g];
    }
    for (int i = 0; i < LUT_N; i++) {
        if (mom) mom[i] = L.mom[i];
        if (var) var[i] = L.var[i];
    }
    if (bias_corr) *bias_corr = L.bias_corr;
    return GS_OK;
}

gs_status gs_set_cull_wait_limit(gs_ctx *c, uint32_t first_wait)
{
    if (!c) {                            // the limit of gs_cull_noalloc (process-wide)
        set_noalloc_first_wait(first_wait);
        return GS_OK;
    }
    c->w.cull_first_wait = first_wait;   // gs_step re-captures its graph when this changes
    return GS_OK;
}

gs_status gs_densify(gs_ctx *c, const gs_scene *src, gs_scene *dst, const gs_adam_cfg *adam, const float *grad_accum,
                     const float *denom, const float *normals, float extent, float grad_threshold,
                     float percent_dense, float min_opacity, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv, dv;
    gs_status st = scene_view(c, src, true, sv);
    if (st) return st;
    if (!valid_adam(adam)) return fail(c, GS_ERR_INVALID_ARG, "invalid adam config");
    sv.opt = adam->optimizer;
    if (src->tier != GS_TIER_DEVICE) return fail(c, GS_ERR_INVALID_ARG, "densification takes a resident scene");
    if (!dst || !grad_accum || !denom || !normals) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    if (!(extent > 0.f) || !std::isfinite(extent) || !std::isfinite(grad_threshold) || !(percent_dense >= 0.f) ||
        !std::isfinite(min_opacity))
        return fail(c, GS_ERR_INVALID_ARG, "invalid densification thresholds");
    if (dst->sh_degree != src->sh_degree || dst->precision != src->precision || dst->tier != GS_TIER_DEVICE ||
        !dst->geo || !dst->sh || !dst->m || !dst->v || !dst->counter || (dst->pitch & 3) || dst->pitch <= 0 ||
        ((src->rdir != nullptr) != (dst->rdir != nullptr)))
        return fail(c, GS_ERR_INVALID_ARG, "destination scene: same degree, precision and planes, resident");
    cudaStream_t s = (cudaStream_t)stream;
    DevArgs a{};
    a.lut = make_lut(adam, src->step + 1, true);
    set_args(c, SLOT_ADAM, a, s);
    uint32_t *masks[3] = {c->amask, c->umask, c->mask};
    uint32_t *prefixes[3] = {c->aprefix, c->wprefix, c->vprefix[0]};
    uint32_t *chunks[3] = {c->achunk, c->uchunk, c->chunk};
    densify_count(sv, c->args + SLOT_ADAM, grad_accum, denom, grad_threshold, percent_dense * extent, min_opacity,
                  masks, prefixes, chunks, c->n_tmp, c->w, s);
    int counts[3] = {0, 0, 0};
    if (cudaMemcpyAsync(counts, c->n_tmp, sizeof(counts), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_check(c, "gs_densify counts");
    const int64_t n_out = (int64_t)counts[0] + counts[1] + 2ll * counts[2];
    dst->n = n_out;
    dst->step = src->step;
    if (n_out > dst->pitch || n_out >= (1ll << 31))
        return fail(c, GS_ERR_CAPACITY, "densified scene has %lld Gaussians, destination pitch %lld",
                    (long long)n_out, (long long)dst->pitch);
    if (n_out == 0) return cuda_check(c, "gs_densify");
    // the destination as the kernels address it (resident planes; it may hold
    // more Gaussians than the context's capacity, which only bounds the source)
    const int64_t eb = elem_bytes(dst->precision), P = dst->pitch;
    dv = sv;
    dv.geo = dst->geo;
    dv.m = dst->m;
    dv.v = dst->v;
    dv.rdir = dst->rdir;
    dv.counter = dst->counter;
    dv.n = n_out;
    dv.pitch = P;
    dv.sh.w = dst->sh;
    dv.sh.m = (char *)dst->m + N_GEO * P * eb;
    dv.sh.v = (char *)dst->v + N_GEO * P * eb;
    dv.sh.rdir = nullptr;
    dv.sh.ppitch = P;
    dv.sh.slot = nullptr;
    densify_write(sv, dv, c->args + SLOT_ADAM, normals, masks, prefixes, c->n_tmp, c->w, s);
    return cuda_check(c, "gs_densify");
}

gs_status gs_step_kernel_count(const gs_ctx *c, int32_t *kernels)
{
    if (!c || !kernels) return GS_ERR_INVALID_ARG;
    *kernels = c->graph.exec ? c->graph.kernels : 0;
    return GS_OK;
}

gs_status gs_render_lists(const gs_ctx *c, const uint32_t **tile_of_key, const uint32_t **splat_of_key,
                          const int32_t **n_keys, const uint32_t **ranges)
{
    if (!c || !c->have_fwd || !tile_of_key || !splat_of_key || !n_keys || !ranges) return GS_ERR_INVALID_ARG;
    *tile_of_key = c->rbs[0].sorted_keys;
    *splat_of_key = c->rbs[0].sorted_vals;
    *n_keys = c->rbs[0].n_keys;
    *ranges = reinterpret_cast<const uint32_t *>(c->rbs[0].ranges);
    return GS_OK;
}

gs_status gs_set_cpu_threads(gs_ctx *c, int32_t threads)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (c->cpu.worker.joinable()) c->cpu.worker.join();
    c->cpu.threads = threads;
    return GS_OK;
}

gs_status gs_cpu_tier_stats(const gs_ctx *c, double *stats)
{
    if (!c || !stats) return GS_ERR_INVALID_ARG;
    const CpuTierState &T = c->cpu;
    const double v[7] = {T.fwd_ms, T.lazy_ms, T.wait_ms, (double)T.h2d, (double)T.d2h, (double)T.rows,
                         (double)T.left};
    for (int i = 0; i < 7; i++) stats[i] = v[i];
    return GS_OK;
}

// Arguments of the host-array optimizer calls (header).
static bool cpu_args_ok(const float *w, const float *m, const float *v, int64_t n_rows, int32_t row, int32_t plane0,
                        int32_t planes, const int32_t *uids, const uint8_t *udelay, int64_t n_upd,
                        const int32_t *vids, const float *grad, int64_t n_vis, int64_t grow,
                        const gs_adam_cfg *adam, int32_t step)
{
    if (!w || !m || !v || n_rows <= 0 || n_rows >= (1ll << 31) || plane0 < 0 || planes < 1 || planes > 64 ||
        row < planes || plane0 + planes > 59)
        return false;
    if (!valid_adam(adam) || adam->mode != GS_ADAM_DEFERRED || step < 0) return false;
    if (n_upd < 0 || n_vis < 0 || (n_upd > 0 && (!uids || !udelay)) || (n_vis > 0 && (!vids || !grad)) ||
        grow < planes)
        return false;
    for (int64_t u = 0; u < n_upd; u++)
        if (uids[u] < 0 || uids[u] >= n_rows || (u && uids[u] <= uids[u - 1]) || udelay[u] > adam->max_defer)
            return false;
    for (int64_t k = 0; k < n_vis; k++)
        if (vids[k] < 0 || vids[k] >= n_rows || (k && vids[k] <= vids[k - 1])) return false;
    return true;
}

static CpuUpdate host_update(const int32_t *uids, const uint8_t *udelay, int64_t n_upd, const int32_t *vids,
                             const float *grad, int64_t n_vis, int64_t grow, const gs_adam_cfg *adam, int32_t step)
{
    CpuUpdate U;
    U.uids = uids;
    U.udelay = udelay;
    U.n_upd = n_upd;
    U.vids = vids;
    U.grad = grad;
    U.n_vis = n_vis;
    U.grow = grow;
    if (step >= 1) U.lut = make_lut(adam, step, true, GS_FP32);
    U.opt = adam->optimizer;
    return U;
}

gs_status gs_cpu_deferred_step(float *w, float *m, float *v, int64_t n_rows, int32_t row, int32_t plane0,
                               int32_t planes, const int32_t *uids, const uint8_t *udelay, int64_t n_upd,
                               const int32_t *vids, const float *grad, int64_t n_vis, int64_t grow,
                               const gs_adam_cfg *adam, int32_t step, int32_t threads)
{
    if (step < 1 || !cpu_args_ok(w, m, v, n_rows, row, plane0, planes, uids, udelay, n_upd, vids, grad, n_vis, grow,
                                 adam, step))
        return GS_ERR_INVALID_ARG;
    cpu_deferred_step(HostPlanes{w, m, v, row, plane0, planes},
                      host_update(uids, udelay, n_upd, vids, grad, n_vis, grow, adam, step), threads);
    return GS_OK;
}

gs_status gs_cpu_forward(const float *w, const float *m, const float *v, int64_t n_rows, int32_t row, int32_t plane0,
                         int32_t planes, const int32_t *ids, const uint8_t *counter, int64_t n, const int32_t *uids,
                         const uint8_t *udelay, int64_t n_upd, const int32_t *vids, const float *grad, int64_t n_vis,
                         int64_t grow, const gs_adam_cfg *adam, int32_t step, float *out, int64_t opitch,
                         int32_t threads)
{
    if (!cpu_args_ok(w, m, v, n_rows, row, plane0, planes, uids, udelay, n_upd, vids, grad, n_vis, grow, adam,
                     step) ||
        n < 0 || (n > 0 && (!ids || !counter || !out)) || opitch < n || (n_upd > 0 && step < 1))
        return GS_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n; k++)
        if (ids[k] < 0 || ids[k] >= n_rows || (k && ids[k] <= ids[k - 1]) || counter[k] > adam->max_defer)
            return GS_ERR_INVALID_ARG;
    const CpuUpdate U = host_update(uids, udelay, n_upd, vids, grad, n_vis, grow, adam, step);
    const DevLut Ln = make_lut(adam, step + 1, true, GS_FP32);
    const HostPlanes P{const_cast<float *>(w), const_cast<float *>(m), const_cast<float *>(v), row, plane0, planes};
    cpu_forward(P, ids, counter, n, n_upd > 0 ? &U : nullptr, Ln, adam->optimizer, out, opitch, threads);
    return GS_OK;
}

gs_status gs_host_tier_stats(const gs_ctx *c, int64_t *chunks, int64_t *bytes)
{
    if (!c || !chunks || !bytes) return GS_ERR_INVALID_ARG;
    *chunks = c->last_touched;
    *bytes = c->last_bytes;
    return GS_OK;
}

gs_status gs_step_gradients(const gs_ctx *c, const float **grad, int64_t *pitch, const int32_t **ids,
                            const int32_t **n)
{
    if (!c || !c->last_views || !grad || !pitch || !ids || !n) return GS_ERR_INVALID_ARG;
    *grad = c->grad_u;
    *pitch = c->last_gpitch;
    *ids = c->last_views > 1 ? c->union_ids : c->vids[0];
    *n = c->last_views > 1 ? &c->cnt->n_union : c->nvis_view;
    return GS_OK;
}

gs_status gs_render_splats(const gs_ctx *c, const float **geom, const float **conic, const int32_t **n_vis)
{
    if (!c || !c->have_fwd || !geom || !conic || !n_vis) return GS_ERR_INVALID_ARG;
    *geom = reinterpret_cast<const float *>(c->rbs[0].rec0);
    *conic = reinterpret_cast<const float *>(c->rbs[0].rec1);
    *n_vis = c->n_render;
    return GS_OK;
}

// ---------------------------------------------------------------------------
// gs_step
struct StepMasks {
    const uint32_t *gmask, *gprefix;   // gradient rows: the view's visible set, or the union of the views'
    int64_t gcap;
    bool selected;                     // the optimizer's select ran inside the cull sweep
};

// Cull of every view (visible ids, counts) and the union of the visible sets.
static StepMasks enqueue_cull_phase(gs_ctx *c, const SceneView &sv, const DevArgs &a, int n_views, float *loss,
                                    cudaStream_t s, int select_max_defer = -1)
{
    const int V = (int)c->cfg.max_visible;
    DevArgs *args = c->args + SLOT_STEP;
    c->w.mark(TP_STEP0, s);
    set_args(c, SLOT_STEP, a, s);
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    const bool selected = select_max_defer >= 0 &&
                          launch_cull_views(sv, args, n_views, c->vmask, c->vchunk, c->w, s, c->umask, c->uchunk,
                                            select_max_defer, &c->cnt->n_cand);
    if (select_max_defer < 0)
        launch_cull_views(sv, args, n_views, c->vmask, c->vchunk, c->w, s, nullptr, nullptr, 0, &c->cnt->n_cand);
    for (int v = 0; v < n_views; v++)
        compact_mask(c->vmask[v], sv.n, c->vchunk[v], true, c->vids[v], c->vprefix[v], V, c->nvis_view + v, c->w, s);
    cudaMemcpyAsync(&c->cnt->n_vis, c->nvis_view, sizeof(int), cudaMemcpyDeviceToDevice, s);
    StepMasks M{c->vmask[0], c->vprefix[0], V, selected};
    if (n_views > 1) {
        const int64_t nw = (sv.n + 31) / 32;
        cudaMemsetAsync(c->union_mask, 0, nw * sizeof(uint32_t), s);
        for (int v = 0; v < n_views; v++) launch_mask_or(c->union_mask, c->vmask[v], nw, c->w, s);
        compact_mask(c->union_mask, sv.n, c->union_chunk, false, c->union_ids, c->union_prefix, (int)c->gcap_u,
                     &c->cnt->n_union, c->w, s);
        M = StepMasks{c->union_mask, c->union_prefix, c->gcap_u, selected};
    }
    c->last_views = n_views;
    c->last_gpitch = M.gcap;
    return M;
}

// Render, L1 loss and backward of every view; gradients summed per Gaussian.
// Views are rendered in rounds of render_slots: each view of a round has its
// lists prepared on the round's buffers; one forward and one backward
// rasterizer launch cover the tiles of the round's views; the projection
// backward of each adds its gradients into the union layout.  The next round
// reuses the same buffers.  (The stage timing points cover the first round.)
static void enqueue_render_phase(gs_ctx *c, const SceneView &sv, const DevArgs &a, int n_views, const StepMasks &M,
                                 float *loss, cudaStream_t s)
{
    DevArgs *args = c->args + SLOT_STEP;
    const int R = render_slots(c->cfg);
    for (int v0 = 0; v0 < n_views; v0 += R) {
        const int k = n_views - v0 < R ? n_views - v0 : R;
        RenderBufs *rbs[MAX_VIEWS];
        const int *nv[MAX_VIEWS];
        const float *dimg_c[MAX_VIEWS];
        for (int j = 0; j < k; j++) {
            rbs[j] = &c->rbs[j];
            nv[j] = c->nvis_view + v0 + j;
            dimg_c[j] = c->dimgs[j];
        }
        if (v0 == 0) c->w.mark(TP_FWD0, s);
        for (int j = 0; j < k; j++)
            prepare_view(sv, args, v0 + j, c->vids[v0 + j], c->nvis_view + v0 + j, c->rbs[j], a.cam[v0 + j], c->w, s,
                         true);
        // the step needs only the final colours the backward reads (no separate image copy)
        float *fin[MAX_VIEWS];
        for (int j = 0; j < k; j++) fin[j] = c->rbs[j].cfinal;
        raster_forward(args, k, rbs, a.cam + v0, fin, true, c->dimgs, loss, c->work, c->w, s, v0);
        if (v0 == 0) {
            c->w.mark(TP_FWD1, s);
            c->w.mark(TP_BWD0, s);
        }
        raster_backward(args, k, rbs, a.cam + v0, dimg_c, nv, c->work + 1, c->w, s, nullptr, v0, true);
        for (int j = 0; j < k; j++) {
            PrevMasks prev{};
            for (int p = 0; p < v0 + j; p++) prev.m[prev.n++] = c->vmask[p];
            project_backward(sv, args, v0 + j, c->nvis_view + v0 + j, c->rbs[j], c->grad_u, M.gcap,
                             n_views > 1 ? M.gmask : nullptr, n_views > 1 ? M.gprefix : nullptr, c->vids[v0 + j],
                             prev, c->w, s);
        }
    }
    c->w.mark(TP_BWD1, s);
}

static void enqueue_adam_phase(gs_ctx *c, const SceneView &sv, int mode, const StepMasks &M, cudaStream_t s)
{
    DevArgs *args = c->args + SLOT_STEP;
    c->w.mark(TP_ADAM0, s);
    if (mode == GS_ADAM_DEFERRED && M.selected && adam_pairs_ok(sv)) {
        launch_adam_pairs(sv, args, M.gmask, M.gprefix, c->grad_u, M.gcap, c->umask, c->uchunk, c->pairs,
                          &c->cnt->n_upd, c->w, s);
    } else if (mode == GS_ADAM_DEFERRED && M.selected) {
        launch_adam_compact(sv, c->umask, c->uchunk, c->uids, c->udelay, &c->cnt->n_upd, c->w, s);
        c->w.mark(TP_APPLY0, s);
        launch_adam_apply(sv, args, M.gmask, M.gprefix, c->grad_u, M.gcap, c->uids, c->udelay, nullptr,
                          &c->cnt->n_upd, c->w, s);
        c->w.mark(TP_APPLY1, s);
    } else if (mode == GS_ADAM_DEFERRED)
        launch_adam_deferred(sv, args, M.gmask, M.gprefix, c->grad_u, M.gcap, c->umask, c->uchunk, c->uids, c->udelay,
                             &c->cnt->n_upd, c->w, s, &c->pairs);
    else
        launch_adam_eager(sv, args, M.gmask, M.gprefix, c->grad_u, M.gcap, c->w, s);
    c->w.mark(TP_ADAM1, s);
    c->w.mark(TP_STEP1, s);
}

// gs_step: the whole iteration enqueued on one stream; captured once into a
// CUDA graph and replayed, with only the argument block (cameras, targets,
// restore tables of the new step) updated between replays.
static void enqueue_step(gs_ctx *c, const SceneView &sv, const DevArgs &a, int n_views, int mode, float *loss,
                         cudaStream_t s)
{
    const StepMasks M = enqueue_cull_phase(c, sv, a, n_views, loss, s,
                                           mode == GS_ADAM_DEFERRED ? a.lut.max_defer : -1);
    if (mode == GS_ADAM_DEFERRED && M.selected && adam_pairs_ok(sv)) {
        // the update set's pairs and delays need only the select: prepared on
        // the side stream during the render (the gather still reads the
        // counters; the apply clears the members')
        const cudaStream_t fs = c->w.fork(s);
        launch_adam_pairs_prep(sv, c->umask, c->uchunk, c->pairs, &c->cnt->n_upd, c->w, fs);
        c->w.side_done(fs);
        enqueue_render_phase(c, sv, a, n_views, M, loss, s);
        DevArgs *args = c->args + SLOT_STEP;
        c->w.mark(TP_ADAM0, s);
        c->w.wait_side(s);
        launch_adam_pairs_apply(sv, args, M.gmask, M.gprefix, c->grad_u, M.gcap, c->pairs, c->w, s);
        c->w.mark(TP_ADAM1, s);
        c->w.mark(TP_STEP1, s);
        return;
    }
    enqueue_render_phase(c, sv, a, n_views, M, loss, s);
    enqueue_adam_phase(c, sv, mode, M, s);
}

// One copy per staged array (w, m, v) of each run of consecutive chunks held
// in consecutive slots: rows [chunk0 << shift, ...) of the host planes <-> the
// slots' rows of the staging ring, all SH planes at once.
static void copy_runs(gs_ctx *c, const gs_scene *scene, const SceneView &sv, size_t first, size_t last, bool to_dev)
{
    const int64_t eb = elem_bytes(scene->precision), R = 1ll << c->shift;
    const int64_t planes = sv.D - N_GEO, ring = sv.sh.ppitch;
    void *host[3] = {scene->host_sh, scene->host_m, scene->host_v};
    for (size_t k = first; k < last; k++) {
        const HostRun &r = c->plan.runs[k];
        const int64_t i0 = r.chunk0 << c->shift;
        const int64_t rows = std::min(sv.n, (r.chunk0 + r.nchunks) << c->shift) - i0;
        for (int j = 0; j < 3; j++) {
            char *h = (char *)host[j] + i0 * eb;
            char *d = (char *)c->stage[j] + r.slot0 * R * eb;
            if (to_dev)
                cudaMemcpy2DAsync(d, ring * eb, h, scene->pitch * eb, rows * eb, planes, cudaMemcpyHostToDevice,
                                  c->cstream);
            else
                cudaMemcpy2DAsync(h, scene->pitch * eb, d, ring * eb, rows * eb, planes, cudaMemcpyDeviceToHost,
                                  c->dstream);
            c->last_bytes += rows * eb * planes;
        }
    }
}

// Device copies of staged chunks from the previous step's slots (w, m, v):
// runs of chunks whose source and destination slots are both consecutive.
static void copy_slots(gs_ctx *c, const gs_scene *scene, const SceneView &sv,
                       const std::vector<std::array<int64_t, 3>> &druns, cudaStream_t s)
{
    const int64_t eb = elem_bytes(scene->precision), R = 1ll << c->shift;
    const int64_t planes = sv.D - N_GEO, ring = sv.sh.ppitch;
    for (const auto &r : druns)                  // {source slot, destination slot, chunks}
        for (int j = 0; j < 3; j++) {
            char *base = (char *)c->stage[j];
            cudaMemcpy2DAsync(base + r[1] * R * eb, ring * eb, base + r[0] * R * eb, ring * eb, r[2] * R * eb, planes,
                              cudaMemcpyDeviceToDevice, s);
        }
}

// gs_step for a host-tier scene (§4.2 selective offloading, SH rows
// streamed).  On the stream: cull and the chunk-touch map, then one host
// synchronisation to read the map.  Chunks with visible Gaussians take the
// first slots of the staging ring for the whole step; the optimizer-only
// chunks (counters at the bound) go through the remaining slots in rounds,
// each round covering a range of chunk ids, alternating between the two
// halves of that part of the ring.  Three streams: the H2D copy stream brings
// the visible chunks (the render waits for these only), then each round's
// chunks once the half it fills has been written back; the stream renders,
// takes the optimizer's select, and per round applies Adam to the members
// whose ids fall in the round's range; the D2H copy stream writes back, after
// each round's apply, that round's chunks and the visible chunks of its id
// range (final from then on).  So the two PCIe directions run at the same
// time.  The last write-backs overlap the next step's cull; that step's
// copies wait for them (ev_end).  Kernels are launched directly (no graph:
// the copies depend on the map).
static gs_status step_host_tier(gs_ctx *c, gs_scene *scene, const SceneView &sv, const DevArgs &a, int n_views,
                                const gs_adam_cfg *adam, float *loss, cudaStream_t s)
{
    if (adam->mode != GS_ADAM_DEFERRED) return fail(c, GS_ERR_INVALID_ARG, "host tier runs the deferred optimizer");
    c->w.capturing = false;
    c->w.tev = c->t_events ? c->t_events + (size_t)c->t_used * TP_COUNT : nullptr;
    struct TevReset {
        gs_ctx *c;
        ~TevReset() { c->w.tev = nullptr; }
    } tev_reset{c};
    const StepMasks M = enqueue_cull_phase(c, sv, a, n_views, loss, s, adam->max_defer);
    if (M.selected)
        launch_touch_from_masks(M.gmask, c->umask, sv.n, c->shift, c->dtouch, c->w, s);
    else
        launch_touch_chunks(M.gmask, sv.counter, sv.n, c->shift, adam->max_defer, c->dtouch, c->w, s);
    const int64_t nch = (sv.n + (1ll << c->shift) - 1) >> c->shift;
    cudaMemcpyAsync(c->htouch, c->dtouch, nch, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "host tier: touch map");
    // the previous step's work is done (at once when it ran on this stream):
    // its slot table copy has landed and its slots hold their final values
    if (cudaEventSynchronize(c->ev_sdone) != cudaSuccess) return cuda_check(c, "host tier: previous step");

    // history of the previous host-tier step on this scene (reset otherwise)
    if (c->pscene != scene->host_sh || c->pn != sv.n || (int64_t)c->hist.pvslot.size() != nch) {
        c->hist.reset(nch);
        c->pscene = scene->host_sh;
        c->pn = sv.n;
    }
    // the plan (host_plan.hpp): ring half, each touched chunk's slot and the
    // source of its rows, the optimizer's rounds, the copy runs
    c->plan = plan_host_step(c->htouch, nch, c->cfg.stage_chunks, c->hist);
    const HostPlan &P = c->plan;
    if (!P.ok)
        return fail(c, GS_ERR_CAPACITY, "host tier: %lld chunks of visible Gaussians, staging ring holds %lld",
                    (long long)P.nv + (P.nu > 0), (long long)c->cfg.stage_chunks);
    const int64_t nv = P.nv, nu = P.nu, nbuf = P.nbuf;
    const bool half = P.half;
    const int p = P.p;
    const std::vector<HostRound> &rounds = P.rounds;
    const std::vector<std::array<int64_t, 3>> &druns = P.druns;
    const size_t now_lo = P.now_lo, late_lo = P.late_lo, late_hi = P.late_hi;
    std::memcpy(c->hslot, P.slot.data(), (size_t)nch * sizeof(int32_t));
    c->last_touched = nv + nu;
    c->last_bytes = 0;
    cudaMemcpyAsync(c->dslot, c->hslot, nch * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaEvent_t prev_done = c->ev_end;            // the previous step's write-backs
    if (P.reuse) {
        // this half was last written back by the step before the previous one
        cudaStreamWaitEvent(c->cstream, c->ev_half[p], 0);
        cudaStreamWaitEvent(s, c->ev_half[p], 0);
        copy_slots(c, scene, sv, druns, s);
    } else {
        cudaStreamWaitEvent(c->cstream, c->ev_end, 0);
    }
    copy_runs(c, scene, sv, now_lo, late_lo, true);
    cudaStreamWaitEvent(c->cstream, prev_done, 0);
    copy_runs(c, scene, sv, late_lo, late_hi, true);
    // the render needs all three arrays (its deferred restore of SH rows reads m and v)
    cudaEventRecord(c->ev_vis, c->cstream);
    cudaStreamWaitEvent(s, c->ev_vis, 0);
    enqueue_render_phase(c, sv, a, n_views, M, loss, s);
    DevArgs *args = c->args + SLOT_STEP;
    c->w.mark(TP_ADAM0, s);
    if (M.selected)
        launch_adam_compact(sv, c->umask, c->uchunk, c->uids, c->udelay, &c->cnt->n_upd, c->w, s);
    else
        launch_adam_select(sv, args, M.gmask, c->umask, c->uchunk, c->uids, c->udelay, &c->cnt->n_upd, c->w, s);
    int *u_range = c->n_tmp + 2;
    const int64_t R = 1ll << c->shift;
    for (size_t k = 0; k < rounds.size(); k++) {
        const HostRound &r = rounds[k];
        // the ring half this round fills was written back by round k - nbuf
        if ((int64_t)k >= nbuf) cudaStreamWaitEvent(c->cstream, c->ev_down[k % nbuf], 0);
        if (r.late) cudaStreamWaitEvent(c->cstream, prev_done, 0);
        copy_runs(c, scene, sv, r.upd_lo, r.upd_hi, true);
        cudaEventRecord(c->ev_upd, c->cstream);
        cudaStreamWaitEvent(s, c->ev_upd, 0);
        launch_uid_range(c->uids, &c->cnt->n_upd, r.ch_lo * R, r.ch_hi * R, u_range, s);
        if (k == 0) c->w.mark(TP_APPLY0, s);
        launch_adam_apply(sv, args, M.gmask, M.gprefix, c->grad_u, M.gcap, c->uids, c->udelay, u_range,
                          &c->cnt->n_upd, c->w, s);
        if (k == 0) c->w.mark(TP_APPLY1, s);
        cudaEventRecord(c->ev_done, s);
        cudaStreamWaitEvent(c->dstream, c->ev_done, 0);
        copy_runs(c, scene, sv, r.upd_lo, r.upd_hi, false);
        copy_runs(c, scene, sv, r.vis_lo, r.vis_hi, false);
        cudaEventRecord(c->ev_down[k % nbuf], c->dstream);
    }
    c->w.mark(TP_ADAM1, s);
    c->w.mark(TP_STEP1, s);
    cudaEventRecord(c->ev_sdone, s);
    cudaEventRecord(c->ev_end, c->dstream);
    if (half) {
        cudaEventRecord(c->ev_half[p], c->dstream);
    } else {
        cudaEventRecord(c->ev_half[0], c->dstream);
        cudaEventRecord(c->ev_half[1], c->dstream);
    }
    advance_host_history(c->hist, c->htouch, nch, P);
    if (c->w.tev) c->t_used++;
    return cuda_check(c, "gs_step host tier");
}

// ---------------------------------------------------------------------------
// GS_TIER_HOST_CPU_OPT: the paper's offloaded configuration with the SH
// optimizer on the host cores (§4.2.2 parameter forwarding, §4.3 deferred
// update with OpenMP).

static double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

static CpuUpdate cpu_update_of(const CpuUpdateBuf &B)
{
    CpuUpdate U;
    U.uids = B.uids;
    U.udelay = B.udelay;
    U.n_upd = B.n_upd;
    U.vids = B.vids;
    U.grad = B.grad;
    U.n_vis = B.n_vis;
    U.grow = B.planes.planes;
    U.lut = B.lut;
    U.opt = B.opt;
    return U;
}

// Apply every held update to its host planes, oldest first (the worker's
// first): the host planes are then the state after the last step.
static gs_status cpu_flush(gs_ctx *c)
{
    CpuTierState &T = c->cpu;
    if (T.worker.joinable()) T.worker.join();
    if (T.down_pending) {
        if (cudaEventSynchronize(T.ev_down) != cudaSuccess) return cuda_check(c, "cpu tier: gradients");
        T.down_pending = false;
    }
    CpuUpdateBuf *order[2] = {&T.buf[0], &T.buf[1]};
    if (order[0]->full && order[1]->full && order[1]->step < order[0]->step) std::swap(order[0], order[1]);
    for (CpuUpdateBuf *B : order)
        if (B->full) {
            cpu_deferred_step(B->planes, cpu_update_of(*B), T.threads);
            B->full = false;
        }
    return GS_OK;
}

// One step.  Host: (A) the worker that applied the update of two steps back is
// joined; (B) after the cull, the visible ids and their counters are read
// (one synchronisation); (C) their SH rows are forwarded from the host planes
// and the previous step's held update into a pinned block, copied to the
// device in pieces as they are ready; (D) a worker thread applies the previous
// step's update to the host planes.  Device (meanwhile): render with the
// forwarded rows, backward, the select and the step of the geometry planes.
// (E) The update-set size and members are read (second synchronisation) and
// the SH gradients copied back on a side stream; they are held for the next
// step.  No graph: the host takes part in every step.
static gs_status step_cpu_tier(gs_ctx *c, gs_scene *scene, const SceneView &sv0, const DevArgs &a, int n_views,
                               const gs_adam_cfg *adam, float *loss, cudaStream_t s)
{
    if (adam->mode != GS_ADAM_DEFERRED) return fail(c, GS_ERR_INVALID_ARG, "the host-core optimizer runs deferred");
    CpuTierState &T = c->cpu;
    const auto t_start = std::chrono::steady_clock::now();
    if (T.worker.joinable()) T.worker.join();                       // (A)
    T.wait_ms = ms_since(t_start);
    const int planes = sv0.D - N_GEO;
    const int64_t G = c->gcap_u;
    const HostPlanes HP{(float *)scene->host_sh, (float *)scene->host_m, (float *)scene->host_v, planes, N_GEO,
                        planes};
    const int32_t t1 = scene->step + 1;
    CpuUpdateBuf &P = T.buf[(t1 - 1) & 1], &B = T.buf[t1 & 1];
    // held updates other than this scene's previous step are applied first
    const bool prev_ours = P.full && P.planes.w == HP.w && P.step == t1 - 1;
    if ((B.full || (P.full && !prev_ours))) {
        if (prev_ours) {
            P.full = false;                     // keep it out of the flush
            const gs_status st = cpu_flush(c);
            P.full = true;
            if (st) return st;
        } else {
            const gs_status st = cpu_flush(c);
            if (st) return st;
        }
    }
    c->w.capturing = false;
    c->w.tev = c->t_events ? c->t_events + (size_t)c->t_used * TP_COUNT : nullptr;
    struct TevReset {
        gs_ctx *c;
        ~TevReset() { c->w.tev = nullptr; }
    } tev_reset{c};
    // (B)
    const StepMasks M = enqueue_cull_phase(c, sv0, a, n_views, loss, s, adam->max_defer);
    const int32_t *vis_d = n_views > 1 ? c->union_ids : c->vids[0];
    const int *nvis_d = n_views > 1 ? &c->cnt->n_union : c->nvis_view;
    launch_gather_u8(sv0.counter, vis_d, nvis_d, (int)M.gcap, T.cnt_d, c->w, s);
    cudaMemcpyAsync(T.counts_h, nvis_d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "cpu tier: visible count");
    const int64_t nv = std::min<int64_t>(std::max(T.counts_h[0], 0), M.gcap);
    cudaMemcpyAsync(B.vids, vis_d, nv * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(T.cnt_h, T.cnt_d, nv, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "cpu tier: visible set");
    if (T.down_pending) {                                            // the previous step's gradients
        if (cudaEventSynchronize(T.ev_down) != cudaSuccess) return cuda_check(c, "cpu tier: gradients");
        T.down_pending = false;
    }
    T.d2h = nv * 5 + 4;
    // (C)
    const CpuUpdate PU = cpu_update_of(P);
    const auto t_fwd = std::chrono::steady_clock::now();
    constexpr int64_t PIECE = 1 << 16;
    for (int64_t k0 = 0; k0 < nv; k0 += PIECE) {
        const int64_t k1 = std::min(nv, k0 + PIECE);
        cpu_forward(HP, B.vids + k0, T.cnt_h + k0, k1 - k0, P.full ? &PU : nullptr, a.lut, adam->optimizer,
                    T.stage_h + k0, G, T.threads);
        cudaMemcpy2DAsync(T.stage_d + k0, G * sizeof(float), T.stage_h + k0, G * sizeof(float),
                          (k1 - k0) * sizeof(float), planes, cudaMemcpyHostToDevice, T.up);
    }
    cudaEventRecord(T.ev_up, T.up);
    T.fwd_ms = ms_since(t_fwd);
    T.rows = nv;
    T.h2d = nv * planes * (int64_t)sizeof(float);
    // (D)
    if (P.full) {
        const int threads = T.threads;
        CpuUpdateBuf *Pp = &P;
        T.worker = std::thread([&T, Pp, threads] {
            const auto t0 = std::chrono::steady_clock::now();
            cpu_deferred_step(Pp->planes, cpu_update_of(*Pp), threads);
            T.lazy_ms = ms_since(t0);
            Pp->full = false;
        });
    } else {
        T.lazy_ms = 0.0;
    }
    // device: render with the forwarded rows, backward, select, geometry step
    cudaStreamWaitEvent(s, T.ev_up, 0);
    SceneView sv = sv0;
    sv.sh.cmask = M.gmask;
    sv.sh.cprefix = M.gprefix;
    enqueue_render_phase(c, sv, a, n_views, M, loss, s);
    DevArgs *args = c->args + SLOT_STEP;
    c->w.mark(TP_ADAM0, s);
    if (M.selected)
        launch_adam_compact(sv, c->umask, c->uchunk, c->uids, c->udelay, &c->cnt->n_upd, c->w, s);
    else
        launch_adam_select(sv, args, M.gmask, c->umask, c->uchunk, c->uids, c->udelay, &c->cnt->n_upd, c->w, s);
    SceneView gv = sv;
    gv.D = N_GEO;                                                    // the geometry planes only
    c->w.mark(TP_APPLY0, s);
    launch_adam_apply(gv, args, M.gmask, M.gprefix, c->grad_u, M.gcap, c->uids, c->udelay, nullptr, &c->cnt->n_upd,
                      c->w, s);
    c->w.mark(TP_APPLY1, s);
    c->w.mark(TP_ADAM1, s);
    c->w.mark(TP_STEP1, s);
    // (E)
    cudaMemcpyAsync(T.counts_h + 1, &c->cnt->n_upd, sizeof(int), cudaMemcpyDeviceToHost, s);
    // SH gradients one row per Gaussian (the host's layout), in the forwarded
    // block (read by this step's gather, which is done)
    launch_to_rows(c->grad_u + (int64_t)N_GEO * M.gcap, M.gcap, planes, nvis_d, (int)M.gcap, T.stage_d, c->w, s);
    cudaEventRecord(T.ev_grad, s);
    cudaStreamWaitEvent(T.down, T.ev_grad, 0);
    cudaMemcpyAsync(B.grad, T.stage_d, nv * planes * sizeof(float), cudaMemcpyDeviceToHost, T.down);
    cudaEventRecord(T.ev_down, T.down);
    T.down_pending = true;
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "cpu tier: update size");
    const int64_t nu = std::min<int64_t>(std::max(T.counts_h[1], 0), sv0.n);
    cudaMemcpyAsync(B.uids, c->uids, nu * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(B.udelay, c->udelay, nu, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "cpu tier: update set");
    B.n_upd = nu;
    B.n_vis = nv;
    B.step = t1;
    B.lut = a.lut;
    B.opt = adam->optimizer;
    B.planes = HP;
    B.full = true;
    T.left = nu;
    T.d2h += nu * 5 + nv * planes * (int64_t)sizeof(float) + 4;
    if (c->w.tev) c->t_used++;
    return cuda_check(c, "gs_step cpu tier");
}

static bool graph_matches(const GraphCache &g, const gs_scene *sc, const gs_camera *views, int n_views, int mode,
                          float *loss, bool timed, int variant, uint32_t first_wait, int opt)
{
    if (!g.exec || g.first_wait != first_wait || g.opt != opt || g.geo != sc->geo || g.sh != sc->sh || g.m != sc->m || g.v != sc->v || g.counter != sc->counter ||
        g.rdir != sc->rdir || g.n != sc->n || g.pitch != sc->pitch || g.deg != sc->sh_degree ||
        g.prec != sc->precision || g.n_views != n_views || g.mode != mode ||
        g.loss != loss || g.timed != timed || g.variant != variant)
        return false;
    for (int v = 0; v < n_views; v++)
        if (g.W[v] != views[v].width || g.H[v] != views[v].height) return false;
    return true;
}

gs_status gs_step(gs_ctx *c, gs_scene *scene, const gs_camera *views, const float *const *targets, int32_t n_views,
                  const gs_adam_cfg *adam, float *loss_out, void *stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    SceneView sv;
    gs_status st = scene_view(c, scene, true, sv, true);
    if (st) return st;
    if (!valid_adam(adam)) return fail(c, GS_ERR_INVALID_ARG, "invalid adam config");
    sv.opt = adam->optimizer;
    if (n_views < 1 || n_views > c->cfg.max_views || !views || !targets || !loss_out)
        return fail(c, GS_ERR_INVALID_ARG, "invalid views/targets/loss");
    DevArgs a{};
    for (int v = 0; v < n_views; v++) {
        if (!valid_cam(c, &views[v]) || !targets[v]) return fail(c, GS_ERR_INVALID_ARG, "invalid view %d", v);
        a.cam[v] = make_cam(views[v], c->cfg.tile_w, c->cfg.tile_h);
        a.target[v] = targets[v];
    }
    a.lut = make_lut(adam, scene->step + 1, adam->mode == GS_ADAM_DEFERRED, scene->precision);
    a.n_views = n_views;
    cudaStream_t s = (cudaStream_t)stream;
    GraphCache &g = c->graph;
    const bool timed = c->t_events != nullptr;
    if (timed && c->t_used >= c->t_max) return fail(c, GS_ERR_CAPACITY, "timing buffer full: call gs_timing_read");
    if (scene->tier == GS_TIER_HOST_SH) {
        st = step_host_tier(c, scene, sv, a, n_views, adam, loss_out, s);
        if (!st) scene->step += 1;
        return st;
    }
    if (scene->tier == GS_TIER_HOST_CPU_OPT) {
        st = step_cpu_tier(c, scene, sv, a, n_views, adam, loss_out, s);
        if (!st) scene->step += 1;
        return st;
    }
    if (!graph_matches(g, scene, views, n_views, adam->mode, loss_out, timed, c->rbs[0].variant * 16 + c->rbs[0].variant_bwd,
                       c->w.cull_first_wait, adam->optimizer)) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        if (g.graph) {
            cudaGraphDestroy(g.graph);
            g.graph = nullptr;
        }
        cudaStream_t cs = s;
        bool own = false;
        if (s == nullptr || s == cudaStreamLegacy) {   // the legacy stream cannot be captured
            cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            own = true;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            if (own) cudaStreamDestroy(cs);
            return cuda_check(c, "gs_step begin capture");
        }
        c->w.tev = timed ? c->t_events : nullptr;        // slot 0 events identify the nodes
        c->w.capturing = true;
        enqueue_step(c, sv, a, n_views, adam->mode, loss_out, cs);
        c->w.capturing = false;
        c->w.tev = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (own) cudaStreamDestroy(cs);
        if (e != cudaSuccess) return fail(c, GS_ERR_CUDA, "gs_step capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return fail(c, GS_ERR_CUDA, "gs_step instantiate: %s", cudaGetErrorString(e));
        }
        // locate the argument-block node
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        cudaGraphNode_t *nodes = (cudaGraphNode_t *)malloc(nn * sizeof(cudaGraphNode_t));
        cudaGraphGetNodes(graph, nodes, &nn);
        g.args_node = nullptr;
        g.kernels = 0;
        for (int p = 0; p < TP_COUNT; p++) g.ev_node[p] = nullptr;
        for (size_t k = 0; k < nn; k++) {
            cudaGraphNodeType ty;
            cudaGraphNodeGetType(nodes[k], &ty);
            if (ty == cudaGraphNodeTypeEventRecord && timed) {
                cudaEvent_t ev;
                cudaGraphEventRecordNodeGetEvent(nodes[k], &ev);
                for (int p = 0; p < TP_COUNT; p++)
                    if (ev == c->t_events[p]) g.ev_node[p] = nodes[k];
                continue;
            }
            if (ty != cudaGraphNodeTypeKernel) continue;
            g.kernels++;
            cudaKernelNodeParams p;
            if (cudaGraphKernelNodeGetParams(nodes[k], &p) == cudaSuccess && p.func == (void *)k_set_args) {
                g.args_node = nodes[k];
                g.args_params = p;
            }
        }
        free(nodes);
        g.graph = graph;
        if (!g.args_node) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            return fail(c, GS_ERR_CUDA, "gs_step: argument node not found");
        }
        g.geo = scene->geo; g.sh = scene->sh; g.m = scene->m; g.v = scene->v; g.counter = scene->counter;
        g.rdir = scene->rdir;
        g.n = scene->n; g.pitch = scene->pitch; g.deg = scene->sh_degree; g.n_views = n_views; g.mode = adam->mode;
        g.prec = scene->precision;
        g.loss = loss_out;
        g.timed = timed;
        g.variant = c->rbs[0].variant * 16 + c->rbs[0].variant_bwd;
        g.first_wait = c->w.cull_first_wait;
        g.opt = adam->optimizer;
        for (int v = 0; v < n_views; v++) { g.W[v] = views[v].width; g.H[v] = views[v].height; }
    }
    if (timed) {
        cudaEvent_t *ev = c->t_events + (size_t)c->t_used * TP_COUNT;
        for (int p = 0; p < TP_COUNT; p++)
            if (g.ev_node[p] && cudaGraphExecEventRecordNodeSetEvent(g.exec, g.ev_node[p], ev[p]) != cudaSuccess)
                return cuda_check(c, "gs_step timing event");
        c->t_used++;
    }
    DevArgs *dst = c->args + SLOT_STEP;
    void *kargs[2] = {&a, &dst};
    cudaKernelNodeParams p = g.args_params;
    p.kernelParams = kargs;
    p.extra = nullptr;
    cudaError_t e = cudaGraphExecKernelNodeSetParams(g.exec, g.args_node, &p);
    if (e != cudaSuccess) return fail(c, GS_ERR_CUDA, "gs_step set args: %s", cudaGetErrorString(e));
    e = cudaGraphLaunch(g.exec, s);
    if (e != cudaSuccess) return fail(c, GS_ERR_CUDA, "gs_step launch: %s", cudaGetErrorString(e));
    scene->step += 1;
    return GS_OK;
}

}  // extern "C"
