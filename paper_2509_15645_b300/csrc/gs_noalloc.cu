// gs_noalloc.cu -- gs_cull_noalloc: the frustum cull without any device
// allocation, for callers that cannot call cudaMalloc (and so cannot create a
// gs_ctx with its own workspace): code running inside a framework whose
// memory pool owns every device byte, loops that forbid allocation after
// start-up, or callers that must keep a fixed, known device footprint.
//
// Its scratch (argument block, visibility bitmask, per-chunk counts, scan
// partials) is one file-scope __device__ array of fixed size, resident on
// every GPU that loads the library until the process exits.  Host code never
// names that array directly: on the first call on each device (with that
// device current) its address is fetched once with cudaGetSymbolAddress and
// cached.  Because of that set-up, the first call on a device should come
// before any stream capture.  All calls share the one array and it keeps the
// last call's contents, so calls that overlap on the GPU (other streams,
// other threads) race; every byte a call reads is written or cleared by that
// same call first (the status word, the bitmask words and chunk counts of the
// scene's range are cleared before the cull, so a cull block that gave up on
// its copies leaves zeros, not the previous call's data).  A status the
// kernels latch (GS_ERR_TIMEOUT) is copied to the caller's status word, and
// the visible count is then 0.
#include <atomic>
#include <mutex>

#include <cmath>

#include "gs_kernels.cuh"

namespace gs {
namespace {

constexpr int64_t NA_MAX = GS_CULL_NOALLOC_MAX_GAUSSIANS;
constexpr int64_t NA_WORDS = NA_MAX / 32 + CHUNK_WORDS;
constexpr int64_t NA_CHUNKS = NA_MAX / CHUNK + 1;

// Byte layout of the scratch array (each part 256-byte aligned).
constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_ARGS = 0;
constexpr size_t OFF_STATUS = round256(OFF_ARGS + sizeof(DevArgs));           // int status, int count
constexpr size_t OFF_PARTIALS = round256(OFF_STATUS + 2 * sizeof(int));
constexpr size_t OFF_CHUNKS = round256(OFF_PARTIALS + 1024 * sizeof(uint32_t));
constexpr size_t OFF_MASK = round256(OFF_CHUNKS + NA_CHUNKS * sizeof(uint32_t));
constexpr size_t SCRATCH_BYTES = round256(OFF_MASK + NA_WORDS * sizeof(uint32_t));

static __device__ __align__(256) unsigned char g_cull_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::atomic<uint32_t> g_first_wait{CULL_WAIT_LIMIT};
std::mutex g_mutex;
unsigned char *g_scratch[MAX_DEVICES] = {nullptr};
int g_sms[MAX_DEVICES] = {0};

__global__ void k_noalloc_args(DevArgs a, DevArgs *dst)
{
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&a);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (int k = threadIdx.x; k < (int)(sizeof(DevArgs) / 4); k += blockDim.x) d[k] = src[k];
}

// After the compaction: the latched status to the caller; an aborted cull
// reports no visible Gaussian.
__global__ void k_noalloc_finish(const int *status, int32_t *status_out, int32_t *n_vis_out)
{
    const int st = *status;
    if (st) *n_vis_out = 0;
    if (status_out) *status_out = st;
}

// Once per device, with that device current: the scratch array's device address.
gs_status scratch_for_current_device(unsigned char **base, int *sms)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cull_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return GS_ERR_CUDA;
        g_scratch[dev] = static_cast<unsigned char *>(p);
        g_sms[dev] = n;
    }
    *base = g_scratch[dev];
    *sms = g_sms[dev];
    return GS_OK;
}

}  // namespace

void set_noalloc_first_wait(uint32_t limit) { g_first_wait.store(limit); }

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_cull_noalloc(const gs_scene *scene, const gs_camera *cam, const gs_adam_cfg *adam,
                                     int32_t tile_w, int32_t tile_h, int32_t *ids_out, int32_t *n_vis_out,
                                     int32_t *status_out, void *stream)
{
    if (!scene || !cam || !ids_out || !n_vis_out || !scene->geo) return GS_ERR_INVALID_ARG;
    if (scene->n <= 0 || scene->pitch < scene->n || (scene->pitch & 3)) return GS_ERR_INVALID_ARG;
    if (scene->n > NA_MAX) return GS_ERR_CAPACITY;     // beyond the fixed scratch: refused, nothing launched
    if (scene->sh_degree < 0 || scene->sh_degree > 3) return GS_ERR_INVALID_ARG;
    if (tile_w <= 0 || tile_h <= 0 || cam->width <= 0 || cam->height <= 0 || !(cam->fx > 0.f) || !(cam->fy > 0.f) ||
        !std::isfinite(cam->fx) || !std::isfinite(cam->fy) || !(cam->far_z > cam->near_z) ||
        cam->width >= 65536 * tile_w || cam->height >= 65536 * tile_h || !camera_region_ok(*cam))
        return GS_ERR_INVALID_ARG;
    if (scene->precision != GS_FP32 && scene->precision != GS_BF16_SH_MOM && scene->precision != GS_BF16_SH_MOM_RN)
        return GS_ERR_INVALID_ARG;
    if (scene->tier != GS_TIER_DEVICE && scene->tier != GS_TIER_HOST_SH) return GS_ERR_INVALID_ARG;
    if (adam && !valid_adam(adam)) return GS_ERR_INVALID_ARG;
    const bool restore = adam && adam->mode == GS_ADAM_DEFERRED && scene->m && scene->v && scene->counter;

    unsigned char *base = nullptr;
    int sms = 0;
    gs_status st = scratch_for_current_device(&base, &sms);
    if (st != GS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // argument block: the camera, and the restore tables of the coming step
    DevArgs a{};
    a.cam[0] = make_cam(*cam, tile_w, tile_h);
    a.n_views = 1;
    if (restore) a.lut = make_lut(adam, scene->step + 1, true);

    DevArgs *args = reinterpret_cast<DevArgs *>(base + OFF_ARGS);
    int *status = reinterpret_cast<int *>(base + OFF_STATUS);
    Work w{};
    w.partials = reinterpret_cast<uint32_t *>(base + OFF_PARTIALS);
    w.status = status;
    w.num_sms = sms;
    w.scan_grid = sms * 2 > 1024 ? 1024 : sms * 2;
    w.tev = nullptr;
    w.cull_first_wait = g_first_wait.load();
    uint32_t *chunks = reinterpret_cast<uint32_t *>(base + OFF_CHUNKS);
    uint32_t *mask = reinterpret_cast<uint32_t *>(base + OFF_MASK);

    SceneView sv{};
    sv.geo = scene->geo;                 // the cull reads the geometry rows only
    sv.tier = scene->tier;
    sv.m = scene->m;
    sv.v = scene->v;
    sv.prec = scene->precision;
    sv.rdir = (scene->m && scene->v) ? scene->rdir : nullptr;
    sv.counter = scene->counter;
    sv.n = scene->n;
    sv.pitch = scene->pitch;
    sv.deg = scene->sh_degree;
    sv.D = N_GEO + 3 * (scene->sh_degree + 1) * (scene->sh_degree + 1);
    sv.opt = adam ? adam->optimizer : GS_OPT_ADAM;

    const int64_t nchunks = (sv.n + CHUNK - 1) / CHUNK;
    k_noalloc_args<<<1, 128, 0, s>>>(a, args);
    cudaMemsetAsync(status, 0, 2 * sizeof(int), s);                 // status and count start at zero
    // a complete cull writes every mask word and chunk count of the range; a
    // block that gives up leaves the cleared values
    cudaMemsetAsync(mask, 0, (size_t)nchunks * CHUNK_WORDS * sizeof(uint32_t), s);
    cudaMemsetAsync(chunks, 0, (size_t)nchunks * sizeof(uint32_t), s);
    launch_cull(sv, args, 0, mask, chunks, w, s);
    compact_mask(mask, sv.n, chunks, true, ids_out, nullptr, (int)sv.n, n_vis_out, w, s);
    k_noalloc_finish<<<1, 1, 0, s>>>(status, status_out, n_vis_out);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
