// k_cull.cu -- frustum cull of every Gaussian (§2.4 step 1, run on the GPU as
// in §4.2.1), plus small bitmask helpers.
//
// One sweep over the geometry planes (mean, log-scale, quaternion: 40 B per
// Gaussian, plus m, v and the counter when the deferred restore of §4.3.3 is
// applied to Gaussians whose counter is non-zero).  Output: one visibility bit
// per Gaussian (warp ballot) and the number of visible Gaussians per
// 2048-Gaussian chunk, from which k_scan.cu builds the ordered id list.
#include <atomic>

#include "gs_kernels.cuh"

namespace gs {

constexpr int CULL_BLOCK = 256;

template <typename MT, int OPT>
__global__ void __launch_bounds__(CULL_BLOCK, 3) k_cull(const float *__restrict__ geo, const MT *__restrict__ m,
                                                     const MT *__restrict__ v, const float *__restrict__ rdir,
                                                     const uint8_t *__restrict__ counter,
                                                     int64_t pitch, int64_t n, const DevArgs *__restrict__ args,
                                                     int view, uint32_t *__restrict__ mask,
                                                     uint32_t *__restrict__ chunk_cnt)
{
    __shared__ DevCam s_cam;
    __shared__ CullCam s_cc;
    __shared__ float s_plut[3][LUT_N], s_dec[3][LUT_N];
    __shared__ float s_eps;
    __shared__ int s_restore;
    __shared__ uint32_t s_cnt[CULL_BLOCK / 32];
    if (threadIdx.x < sizeof(DevCam) / 4)
        ((uint32_t *)&s_cam)[threadIdx.x] = ((const uint32_t *)&args->cam[view])[threadIdx.x];
    if (threadIdx.x == 0) make_cull_cam(args->cam[view], s_cc);
    if (threadIdx.x < 3 * LUT_N) {
        s_plut[threadIdx.x / LUT_N][threadIdx.x % LUT_N] = args->lut.param[threadIdx.x / LUT_N][threadIdx.x % LUT_N];
        s_dec[threadIdx.x / LUT_N][threadIdx.x % LUT_N] = args->lut.decay[threadIdx.x / LUT_N][threadIdx.x % LUT_N];
    }
    if (threadIdx.x == 0) {
        s_eps = args->lut.eps;
        s_restore = args->lut.restore && m != nullptr && v != nullptr && counter != nullptr;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nchunks = (n + CHUNK - 1) / CHUNK;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        uint32_t cnt = 0;
#pragma unroll 1
        for (int j = 0; j < CHUNK / CULL_BLOCK; j++) {
            int64_t wbase = c * CHUNK + j * CULL_BLOCK + wid * 32;
            int64_t i = wbase + lane;
            int keep = 0;
            if (i < n) {
                float g[10];
#pragma unroll
                for (int r = 0; r < 10; r++) g[r] = __ldg(geo + r * pitch + i);
                if (s_restore && rdir) {
                    // restore through the stored directions: w and dir loads issued together
                    float dd[10];
#pragma unroll
                    for (int r = 0; r < 10; r++) dd[r] = __ldg(rdir + r * pitch + i);
                    const int d = counter[i];
#pragma unroll
                    for (int r = 0; r < 10; r++)
                        g[r] = restore_with_dir<OPT>(g[r], dd[r], s_plut[lr_group(r)][d], s_dec[lr_group(r)][d], d);
                } else if (s_restore) {
                    // m, v loads are issued together with w, not after the counter arrives
                    float mm[10], vv[10];
#pragma unroll
                    for (int r = 0; r < 10; r++) {
                        mm[r] = ld_val(m + r * pitch + i);
                        vv[r] = ld_val(v + r * pitch + i);
                    }
                    const int d = counter[i];
#pragma unroll
                    for (int r = 0; r < 10; r++)
                        g[r] = restore_param<OPT>(g[r], mm[r], vv[r], s_plut[lr_group(r)][d], s_dec[lr_group(r)][d], d,
                                                  s_eps);
                }
                if (maybe_visible(g, s_cc)) {
                    Proj P;
                    project_gaussian(g, s_cam, P);
                    keep = P.keep;
                }
            }
            uint32_t word = __ballot_sync(0xffffffffu, keep);
            if (lane == 0 && wbase < n) {
                mask[wbase >> 5] = word;
                cnt += __popc(word);
            }
        }
        if (lane == 0) s_cnt[wid] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int k = 0; k < CULL_BLOCK / 32; k++) t += s_cnt[k];
            chunk_cnt[c] = t;
        }
        __syncthreads();
    }
}

// The same cull with the planes staged in shared memory by the TMA engine:
// tiles of CT Gaussians, each the CT-element segments of the 10 geometry
// planes and (restoring) their 10 restore-direction planes, in a ring of
// CSTAGES buffers, so HBM streams independently of how many warps are
// resident.  Thread 0 issues the bulk copies CSTAGES - 1 tiles ahead; every
// thread waits on the tile's barrier (bounded: on a timeout the block latches
// GS_ERR_TIMEOUT and stops after draining what it issued).  The first wait of
// each block has its own limit `first_wait` (CULL_WAIT_LIMIT unless a test
// lowers it to make the timeout path run; the drain always uses the full
// limit, so the copies in flight land before the block exits).
// The stages hold the planes every Gaussian needs (mean and log-scale, 0-5)
// with their restore directions; the rotation planes (6-9) are read directly
// for the Gaussians that pass the pre-test.  A tile is TT = 512 Gaussians; each
// of the CT = 256 threads takes two of them (tid and tid + 256), so the tile's
// fixed costs are shared by twice the work and the two chains interleave.  The
// kernel is bound by latency, not bandwidth: two stages (one tile landing while
// the other is consumed) leave room for four blocks (32 warps) per SM, which
// measured faster than three stages at two or three blocks.
constexpr int CT = 256, CG = 2, TT = CT * CG, CSTAGES = 2, CPLANES = 10, CPRE = 6;
struct CullStage {
    float geo[CPRE][TT];
    float dir[CPRE][TT];
    uint8_t cnt[TT];      // counters of a full tile (the last, partial tile reads them directly)
};
constexpr size_t CULL_SMEM = sizeof(CullStage) * CSTAGES;
constexpr uint32_t WAIT_LIMIT = CULL_WAIT_LIMIT;

// Views [view0, view0 + nv) of the argument block in one sweep: the planes
// are read and restored once and projected into every view.
struct CullOut {
    uint32_t *mask[MAX_VIEWS];
    uint32_t *chunk[MAX_VIEWS];
    // optional, inside a training step: the deferred optimizer's select of
    // Fig. 10 on the same sweep -- update-set mask (visible in some view, or
    // counter at max_defer), per-chunk member counts, counters of the other
    // Gaussians incremented
    uint32_t *umask;
    uint32_t *uchunk;
    uint8_t *counter_rw;
    int *n_cand;          // optional: number of Gaussians whose rotation planes were read
};

// ONE: a single view (nv == 1), compiled with the view loop removed.
template <int OPT, bool ONE>
__global__ void __launch_bounds__(CT, 4) k_cull_tma(const float *__restrict__ geo, const float *__restrict__ rdir,
                                                   const uint8_t *__restrict__ counter, int64_t pitch, int64_t n,
                                                   const DevArgs *__restrict__ args, int view0, int nv_arg,
                                                   const CullOut out, int *status, uint32_t first_wait)
{
    const int nv = ONE ? 1 : nv_arg;
    extern __shared__ __align__(128) unsigned char smem[];
    CullStage *st = reinterpret_cast<CullStage *>(smem);
    __shared__ __align__(8) uint64_t bar[CSTAGES];
    __shared__ DevCam s_cam[MAX_VIEWS];
    __shared__ CullCam s_cc[MAX_VIEWS];
    __shared__ float s_plut[3][LUT_N], s_dec[3][LUT_N];
    __shared__ uint32_t s_cnt[MAX_VIEWS][CT / 32];
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < nv * (int)(sizeof(DevCam) / 4); e += CT) {
        const int v = e / (int)(sizeof(DevCam) / 4), o = e % (int)(sizeof(DevCam) / 4);
        ((uint32_t *)&s_cam[v])[o] = ((const uint32_t *)&args->cam[view0 + v])[o];
    }
    if (tid < nv) make_cull_cam(args->cam[view0 + tid], s_cc[tid]);
    if (tid < MAX_VIEWS * (CT / 32)) s_cnt[tid / (CT / 32)][tid % (CT / 32)] = 0;
    if (tid < 3 * LUT_N) {
        s_plut[tid / LUT_N][tid % LUT_N] = args->lut.param[tid / LUT_N][tid % LUT_N];
        s_dec[tid / LUT_N][tid % LUT_N] = args->lut.decay[tid / LUT_N][tid % LUT_N];
    }
    const bool restore = args->lut.restore && rdir != nullptr && counter != nullptr;
    const bool select = out.umask != nullptr;
    const bool need_cnt = restore || select;
    const int max_defer = args->lut.max_defer;
    if (tid == 0) {
        s_abort = 0;
        for (int k = 0; k < CSTAGES; k++) mbar_init(&bar[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    constexpr int PER_CHUNK = CHUNK / TT;
    static_assert(CHUNK % TT == 0, "a chunk is a whole number of tiles");
    const int64_t ntiles = (n + TT - 1) / TT, nchunks = (n + CHUNK - 1) / CHUNK;
    // q-th tile of this block (chunks blockIdx.x, + gridDim.x, ...), or -1
    auto tile_of = [&](int64_t q) -> int64_t {
        const int64_t c = blockIdx.x + (q / PER_CHUNK) * gridDim.x;
        if (c >= nchunks) return -1;
        const int64_t t = c * PER_CHUNK + q % PER_CHUNK;
        return t < ntiles ? t : -1;
    };
    auto issue = [&](int64_t q) {                  // thread 0 only
        const int64_t t = tile_of(q);
        if (t < 0) return;
        const int s = (int)(q % CSTAGES);
        const int64_t i0 = t * TT;
        const int64_t rows = min((int64_t)TT, n - i0);
        const uint32_t bytes = (uint32_t)(((rows + 3) & ~3ll) * 4);   // within the plane: pitch >= n, a multiple of 4
        const bool cnt_bulk = need_cnt && rows == TT;
        mbar_expect_tx(&bar[s], bytes * CPRE * (restore ? 2u : 1u) + (cnt_bulk ? (uint32_t)TT : 0u));
        for (int r = 0; r < CPRE; r++) bulk_g2s(st[s].geo[r], geo + r * pitch + i0, bytes, &bar[s]);
        if (restore)
            for (int r = 0; r < CPRE; r++) bulk_g2s(st[s].dir[r], rdir + r * pitch + i0, bytes, &bar[s]);
        if (cnt_bulk) bulk_g2s(st[s].cnt, counter + i0, TT, &bar[s]);
    };
    if (tid == 0)
        for (int q = 0; q < CSTAGES - 1; q++) issue(q);
    int64_t issued_to = CSTAGES - 1;               // tiles [0, issued_to) issued (thread 0's view)
    int64_t q_stop = 0;                            // first tile not consumed when the loop ends
    uint32_t n_full = 0;                           // Gaussians of this thread whose rotation planes were read
    for (int64_t q = 0;; q++) {
        q_stop = q;
        const int64_t c = blockIdx.x + (q / PER_CHUNK) * gridDim.x;
        if (c >= nchunks) break;
        if (tid == 0) {
            issue(q + CSTAGES - 1);                // into the buffer freed at the end of tile q - 1
            issued_to = q + CSTAGES;
        }
        const int64_t t = tile_of(q);
        if (t >= 0) {
            const int s = (int)(q % CSTAGES);
            if (!mbar_wait_bounded(&bar[s], (uint32_t)((q / CSTAGES) & 1), q == 0 ? first_wait : WAIT_LIMIT))
                s_abort = 1;
            const bool full_tile = t * TT + TT <= n;
            // planes 0-5 (mean, log-scale) of both Gaussians from the stage: the
            // pre-test needs only those; the rotation planes are read for its survivors
            float g[CG][CPLANES];
            int d[CG];
            bool live[CG], full[CG], any_view[CG];
#pragma unroll
            for (int e = 0; e < CG; e++) {
                const int k = tid + e * CT;
                const int64_t i = t * TT + k;
                live[e] = i < n && !s_abort;
                full[e] = false;
                any_view[e] = false;
#pragma unroll
                for (int r = 0; r < CPRE; r++) g[e][r] = live[e] ? st[s].geo[r][k] : 0.f;
                d[e] = (need_cnt && live[e]) ? (full_tile ? st[s].cnt[k] : counter[i]) : 0;
            }
            if (restore) {
#pragma unroll
                for (int e = 0; e < CG; e++) {
                    const int k = tid + e * CT;
#pragma unroll
                    for (int r = 0; r < CPRE; r++)
                        if (live[e])
                            g[e][r] = restore_with_dir<OPT>(g[e][r], st[s].dir[r][k], s_plut[lr_group(r)][d[e]],
                                                            s_dec[lr_group(r)][d[e]], d[e]);
                }
            }
            for (int v = 0; v < nv; v++) {
                bool mv[CG];
#pragma unroll
                for (int e = 0; e < CG; e++) mv[e] = live[e] && maybe_visible(g[e], s_cc[v]);   // most leave here
#pragma unroll
                for (int e = 0; e < CG; e++) {
                    int keep = 0;
                    const int64_t i = t * TT + tid + e * CT;
                    if (mv[e]) {
                        if (!full[e]) {
#pragma unroll
                            for (int r = CPRE; r < CPLANES; r++) g[e][r] = __ldg(geo + r * pitch + i);
                            if (restore && d[e]) {
                                float dd[CPLANES - CPRE];
#pragma unroll
                                for (int r = CPRE; r < CPLANES; r++) dd[r - CPRE] = __ldg(rdir + r * pitch + i);
#pragma unroll
                                for (int r = CPRE; r < CPLANES; r++)
                                    g[e][r] = restore_with_dir<OPT>(g[e][r], dd[r - CPRE], s_plut[lr_group(r)][d[e]],
                                                                    s_dec[lr_group(r)][d[e]], d[e]);
                            }
                            full[e] = true;
                            n_full++;
                        }
                        Proj P;
                        project_gaussian(g[e], s_cam[v], P);
                        keep = P.keep;
                    }
                    any_view[e] |= keep != 0;
                    const uint32_t word = __ballot_sync(0xffffffffu, keep);
                    const int64_t wbase = t * TT + e * CT + wid * 32;
                    if (lane == 0 && wbase < n) {
                        out.mask[v][wbase >> 5] = word;
                        s_cnt[v][wid] += __popc(word);
                    }
                }
            }
            if (select) {
#pragma unroll
                for (int e = 0; e < CG; e++) {
                    const int64_t i = t * TT + tid + e * CT;
                    const bool in_u = live[e] && (any_view[e] || d[e] >= max_defer);
                    if (live[e] && !in_u) out.counter_rw[i] = (uint8_t)(d[e] + 1);
                    const uint32_t uword = __ballot_sync(0xffffffffu, in_u);
                    const int64_t wbase = t * TT + e * CT + wid * 32;
                    if (lane == 0 && wbase < n) {
                        out.umask[wbase >> 5] = uword;
                        if (uword) atomicAdd(&out.uchunk[t / PER_CHUNK], (uint32_t)__popc(uword));
                    }
                }
            }
        }
        __syncthreads();                           // buffer q % CSTAGES is free again
        if (s_abort) break;                        // q_stop = q: its copy may still be landing
        if (q % PER_CHUNK == PER_CHUNK - 1) {      // the chunk's counts (s_cnt settled by the barrier above)
            if (tid < nv) {
                uint32_t tot = 0;
                for (int k = 0; k < CT / 32; k++) {
                    tot += s_cnt[tid][k];
                    s_cnt[tid][k] = 0;
                }
                out.chunk[tid][c] = tot;
            }
            __syncthreads();                       // counts cleared before the next tile adds to them
        }
    }
    if (out.n_cand) {
#pragma unroll
        for (int o = 16; o; o >>= 1) n_full += __shfl_xor_sync(0xffffffffu, n_full, o);
        if (lane == 0 && n_full) atomicAdd(out.n_cand, (int)n_full);
    }
    if (s_abort) {
        // the block's chunks from the one it stopped in onwards: no visible
        // Gaussian and no update-set member (mask words and counts cleared), so
        // the compactions that follow see a consistent, smaller set
        const int64_t nwords = (n + 31) >> 5;
        for (int64_t c = blockIdx.x + (q_stop / PER_CHUNK) * gridDim.x; c < nchunks; c += gridDim.x) {
            const int64_t w1 = min(nwords, (c + 1) * (int64_t)CHUNK_WORDS);
            for (int64_t wd = c * CHUNK_WORDS + tid; wd < w1; wd += CT) {
                for (int v = 0; v < nv; v++) out.mask[v][wd] = 0u;
                if (select) out.umask[wd] = 0u;
            }
            if (tid < nv) out.chunk[tid][c] = 0u;
            if (select && tid == 0) out.uchunk[c] = 0u;
        }
    }
    if (s_abort && tid == 0) {
        latch(status, GS_ERR_TIMEOUT);
        // let the copies this block issued and did not consume land before its
        // shared memory goes away (at most CSTAGES - 1 tiles)
        for (int64_t q = q_stop; q < issued_to; q++)
            if (tile_of(q) >= 0) mbar_wait_bounded(&bar[q % CSTAGES], (uint32_t)((q / CSTAGES) & 1), WAIT_LIMIT);
    }
}

static bool cull_tma_ok(const SceneView &sc)
{
    const bool restore_dir_path = sc.rdir != nullptr || !(sc.m && sc.v && sc.counter);
    const bool aligned = ((uintptr_t)sc.geo & 15) == 0 && ((uintptr_t)sc.rdir & 15) == 0 &&
                         ((uintptr_t)sc.counter & 15) == 0;   // bulk-copy rule
    return restore_dir_path && aligned;
}

template <int OPT>
static void launch_cull_tma_t(const SceneView &sc, const DevArgs *args, int view0, int nv, const CullOut &out, Work &w,
                              cudaStream_t s)
{
    // the stages exceed the default dynamic shared-memory limit; the raised
    // limit is a per-device setting, recorded per device (and per instance)
    static std::atomic<uint64_t> attr_devices{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(attr_devices.load() & bit)) {
        cudaFuncSetAttribute(k_cull_tma<OPT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CULL_SMEM);
        cudaFuncSetAttribute(k_cull_tma<OPT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CULL_SMEM);
        attr_devices.fetch_or(bit);
    }
    const int64_t nchunks = (sc.n + CHUNK - 1) / CHUNK;
    if (out.umask) cudaMemsetAsync(out.uchunk, 0, (size_t)nchunks * sizeof(uint32_t), s);   // atomics
    if (out.n_cand) cudaMemsetAsync(out.n_cand, 0, sizeof(int), s);
    const int gt = w.grid(nchunks * CT, CT, 4);
    (nv == 1 ? k_cull_tma<OPT, true> : k_cull_tma<OPT, false>)<<<gt, CT, CULL_SMEM, s>>>(
        sc.geo, sc.rdir, sc.counter, sc.pitch, sc.n, args, view0, nv, out, w.status, w.cull_first_wait);
}

// The restore through stored directions differs between optimizers only by
// AdamW's decay: Adam and momentum SGD share one instance.
static void launch_cull_tma(const SceneView &sc, const DevArgs *args, int view0, int nv, const CullOut &out, Work &w,
                            cudaStream_t s)
{
    if (sc.opt == GS_OPT_ADAMW) launch_cull_tma_t<GS_OPT_ADAMW>(sc, args, view0, nv, out, w, s);
    else launch_cull_tma_t<GS_OPT_ADAM>(sc, args, view0, nv, out, w, s);
}

void launch_cull(const SceneView &sc, const DevArgs *args, int view, uint32_t *mask, uint32_t *chunk_cnt, Work &w,
                 cudaStream_t s)
{
    int64_t nchunks = (sc.n + CHUNK - 1) / CHUNK;
    if (view == 0) w.mark(TP_CULL0, s);
    const int g = w.grid(nchunks * CULL_BLOCK, CULL_BLOCK, 8);
    if (cull_tma_ok(sc)) {
        // geometry (and restore directions) staged by the TMA engine
        CullOut out{};
        out.mask[0] = mask;
        out.chunk[0] = chunk_cnt;
        launch_cull_tma(sc, args, view, 1, out, w, s);
    } else {
        with_opt(sc.opt, [&](auto o) {
            constexpr int OPT = decltype(o)::value;
            if (sc.prec == GS_FP32)
                k_cull<float, OPT><<<g, CULL_BLOCK, 0, s>>>(sc.geo, (const float *)sc.m, (const float *)sc.v, sc.rdir,
                                                            sc.counter, sc.pitch, sc.n, args, view, mask, chunk_cnt);
            else
                k_cull<__nv_bfloat16, OPT><<<g, CULL_BLOCK, 0, s>>>(sc.geo, (const __nv_bfloat16 *)sc.m,
                                                                    (const __nv_bfloat16 *)sc.v, sc.rdir, sc.counter,
                                                                    sc.pitch, sc.n, args, view, mask, chunk_cnt);
        });
    }
    if (view == 0) w.mark(TP_CULL1, s);
}

bool launch_cull_views(const SceneView &sc, const DevArgs *args, int n_views, uint32_t *const *masks,
                       uint32_t *const *chunk_cnts, Work &w, cudaStream_t s, uint32_t *umask, uint32_t *uchunk,
                       int max_defer, int *n_cand)
{
    if (!cull_tma_ok(sc)) {
        for (int v = 0; v < n_views; v++) launch_cull(sc, args, v, masks[v], chunk_cnts[v], w, s);
        return false;                              // the optimizer's select stays a pass of its own
    }
    w.mark(TP_CULL0, s);
    CullOut out{};
    for (int v = 0; v < n_views; v++) {
        out.mask[v] = masks[v];
        out.chunk[v] = chunk_cnts[v];
    }
    out.n_cand = n_cand;
    if (umask && sc.counter) {
        out.umask = umask;
        out.uchunk = uchunk;
        out.counter_rw = sc.counter;
        (void)max_defer;                           // the kernel reads the step's bound from the argument block
    }
    launch_cull_tma(sc, args, 0, n_views, out, w, s);
    w.mark(TP_CULL1, s);
    return out.umask != nullptr;
}

// Build a bitmask from an id list (ids < n).
__global__ void k_ids_to_mask(const int32_t *__restrict__ ids, const int *n_dev, int cap, uint32_t *mask, int64_t n)
{
    int cnt = *n_dev;
    if (cnt > cap) cnt = cap;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        int i = ids[k];
        if (i >= 0 && i < n) atomicOr(mask + (i >> 5), 1u << (i & 31));
    }
}

void launch_ids_to_mask(const int32_t *ids, const int *n_dev, int cap, uint32_t *mask, int64_t n, Work &w,
                        cudaStream_t s)
{
    cudaMemsetAsync(mask, 0, ((n + 31) / 32) * sizeof(uint32_t), s);
    k_ids_to_mask<<<w.grid(cap, 256), 256, 0, s>>>(ids, n_dev, cap, mask, n);
}

__global__ void k_mask_or(uint32_t *dst, const uint32_t *__restrict__ src, int64_t nwords)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nwords; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] |= src[k];
}

void launch_mask_or(uint32_t *dst, const uint32_t *src, int64_t nwords, Work &w, cudaStream_t s)
{
    k_mask_or<<<w.grid(nwords, 256), 256, 0, s>>>(dst, src, nwords);
}

}  // namespace gs
