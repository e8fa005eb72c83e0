// k_adam.cu -- the optimizer step of GS-Scale §4.3 on the GPU.
//
// Deferred Adam (Eqs. 2-3, pseudocode of Fig. 10): the update set is the
// Gaussians with a gradient this step plus those whose 4-bit counter reached
// MAX.  Members are restored through the tables (param_lut, mom_lut, var_lut)
// and stepped with Eq. 1; every other counter is incremented.  The paper runs
// this loop on the CPU with OpenMP over update_ids; here it is two HBM sweeps:
//   k_adam_select  -- counters (1 B) + visibility mask: update-set bitmask,
//                     counters of non-members incremented in place;
//   k_compact      -- ordered id list of the update set (k_scan.cu);
//   k_adam_apply   -- one thread per (member, 4 planes), w, m, v (+ g) and the
//                     restore direction: 28 B read/written per parameter in
//                     the fp32 form, 14 B per SH parameter in the bf16 form;
//                     coalesced because the Gaussians are stored in Morton
//                     order and views see runs.
#include <type_traits>

#include "gs_kernels.cuh"

namespace gs {

constexpr int ADAM_BLOCK = 256;

__global__ void __launch_bounds__(ADAM_BLOCK) k_adam_select(uint8_t *__restrict__ counter,
                                                            const uint32_t *__restrict__ vmask, int64_t n,
                                                            const DevArgs *__restrict__ args,
                                                            uint32_t *__restrict__ umask,
                                                            uint32_t *__restrict__ uchunk)
{
    __shared__ uint32_t s_cnt[ADAM_BLOCK / 32];
    const int max_defer = args->lut.max_defer;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nchunks = (n + CHUNK - 1) / CHUNK;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        uint32_t cnt = 0;
#pragma unroll 2
        for (int j = 0; j < CHUNK / ADAM_BLOCK; j++) {
            int64_t wbase = c * CHUNK + j * ADAM_BLOCK + wid * 32;
            int64_t i = wbase + lane;
            bool in_u = false;
            uint32_t vw = 0;
            if (wbase < n) vw = vmask[wbase >> 5];
            if (i < n) {
                int cv = counter[i];
                bool vis = (vw >> lane) & 1u;
                in_u = vis || cv >= max_defer;
                if (!in_u) counter[i] = (uint8_t)(cv + 1);
            }
            uint32_t word = __ballot_sync(0xffffffffu, in_u);
            if (lane == 0 && wbase < n) {
                umask[wbase >> 5] = word;
                cnt += __popc(word);
            }
        }
        if (lane == 0) s_cnt[wid] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int k = 0; k < ADAM_BLOCK / 32; k++) t += s_cnt[k];
            uchunk[c] = t;
        }
        __syncthreads();
    }
}

// Host tier (§4.2 selective offloading): which chunks of 2^shift Gaussians
// this step touches.  touch[c] = 2 if a Gaussian of chunk c is visible (its SH
// rows feed the gather and the optimizer), 1 if one is only in the update set
// (its counter reached max_defer), else 0 -- the same membership test as
// k_adam_select, taken before the counters change.
__global__ void __launch_bounds__(ADAM_BLOCK) k_touch_chunks(const uint32_t *__restrict__ vmask,
                                                             const uint8_t *__restrict__ counter, int64_t n, int shift,
                                                             int max_defer, uint8_t *__restrict__ touch)
{
    const int64_t R = 1ll << shift, nchunks = (n + R - 1) >> shift;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t i0 = c << shift, i1 = min(n, i0 + R);
        int vis = 0, sat = 0;
        for (int64_t wd = (i0 >> 5) + threadIdx.x; wd < ((i1 + 31) >> 5); wd += blockDim.x) vis |= vmask[wd] != 0u;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) sat |= counter[i] >= max_defer;
        vis = __syncthreads_or(vis);
        sat = __syncthreads_or(sat);
        if (threadIdx.x == 0) touch[c] = vis ? 2 : (sat ? 1 : 0);
    }
}

void launch_touch_chunks(const uint32_t *vmask, const uint8_t *counter, int64_t n, int shift, int max_defer,
                         uint8_t *touch, Work &w, cudaStream_t s)
{
    const int64_t nchunks = (n + (1ll << shift) - 1) >> shift;
    k_touch_chunks<<<w.grid(nchunks * ADAM_BLOCK, ADAM_BLOCK, 4), ADAM_BLOCK, 0, s>>>(vmask, counter, n, shift,
                                                                                   max_defer, touch);
}

// Shared copy of the step's tables.
struct SLut {
    float param[N_GROUPS][LUT_N];
    float decay[N_GROUPS][LUT_N];
    float mom[LUT_N], var[LUT_N];
    float step_size[N_GROUPS], wdf[N_GROUPS];
    float bias_corr, inv_bias_corr, omb1, omb2, eps;
    uint32_t seed, step;
    int stochastic;
};

__device__ __forceinline__ void load_slut(SLut &s, const DevLut &L)
{
    int t = threadIdx.x;
    if (t < N_GROUPS * LUT_N) {
        s.param[t / LUT_N][t % LUT_N] = L.param[t / LUT_N][t % LUT_N];
        s.decay[t / LUT_N][t % LUT_N] = L.decay[t / LUT_N][t % LUT_N];
    }
    if (t < LUT_N) { s.mom[t] = L.mom[t]; s.var[t] = L.var[t]; }
    if (t < N_GROUPS) {
        s.step_size[t] = L.step_size[t];
        s.wdf[t] = L.wdf[t];
    }
    if (t == 0) {
        s.bias_corr = L.bias_corr;
        s.inv_bias_corr = L.inv_bias_corr;
        s.omb1 = L.omb1;
        s.omb2 = L.omb2;
        s.eps = L.eps;
        s.seed = L.seed;
        s.step = (uint32_t)L.step;
        s.stochastic = L.stochastic;
    }
    __syncthreads();
}

// Restore (delay d) + one optimizer step for one value; d = 0 is the plain
// step.  Adam: Eq. 1.  AdamW: Eq. 1 after the decoupled decay of the step
// (wdf = 1 - lr wd) and with the deferred steps' decay in the restore.
// Momentum SGD: the buffer lives in m (mom = mu^(d+1), omb1 = 1), v is left
// alone.
template <int OPT>
__device__ __forceinline__ void adam_value(float &w, float &m, float &v, float g, int d, int grp, const SLut &L)
{
    const float m_new = L.mom[d] * m + L.omb1 * g;
    if (OPT == GS_OPT_SGDM) {
        const float wr = restore_param<OPT>(w, m, v, L.param[grp][d], 1.f, d, L.eps);
        w = wr - L.step_size[grp] * m_new;
        m = m_new;
        return;
    }
    const float v_new = L.var[d] * v + L.omb2 * g * g;
    const float wr = restore_param<OPT>(w, m, v, L.param[grp][d], L.decay[grp][d], d, L.eps);
    const float denom = sqrt_fast(v_new) * L.inv_bias_corr + L.eps;
    const float ws = OPT == GS_OPT_ADAMW ? __fmul_rn(L.wdf[grp], wr) : wr;
    w = ws - L.step_size[grp] * __fdividef(m_new, denom);
    m = m_new;
    v = v_new;
}

__device__ __forceinline__ int compact_index(const uint32_t *__restrict__ vmask, const uint32_t *__restrict__ vprefix,
                                             int64_t i)
{
    uint32_t word = vmask[i >> 5];
    uint32_t bit = (uint32_t)(i & 31);
    if (!((word >> bit) & 1u)) return -1;
    return (int)(vprefix[i >> 5] + __popc(word & ((1u << bit) - 1u)));
}

// Parameter plane r of Gaussian i: the 11 geometry planes (w fp32, m and v of
// type T, restore direction fp32) at r * pitch + i; SH plane r (w, m, v and
// restore direction of type T) at (r - 11) * sp + sb, where sb = shbase(i) is
// i for a resident scene and the staging-ring element for the host tier.
template <typename T, typename IX = int64_t> struct Planes {
    float *geo;
    T *m, *v;
    float *rdir;
    T *shw, *shm, *shv;
    IX pitch, sp;
    const int32_t *slot;
    int shift;
    __device__ __forceinline__ IX shbase(IX i) const
    {
        if (!slot) return i;
        return ((IX)max(__ldg(slot + (i >> shift)), 0) << shift) + (i & (((IX)1 << shift) - 1));
    }
    __device__ __forceinline__ IX go(int r, IX i) const { return (IX)r * pitch + i; }
    __device__ __forceinline__ IX so(int r, IX sb) const { return (IX)(r - N_GEO) * sp + sb; }
    __device__ __forceinline__ float ldw(int r, IX i, IX sb) const
    {
        return r < N_GEO ? geo[go(r, i)] : ld_val(shw + so(r, sb));
    }
    __device__ __forceinline__ float ldm(int r, IX i, IX sb) const
    {
        return ld_val(r < N_GEO ? m + go(r, i) : shm + so(r, sb));
    }
    __device__ __forceinline__ float ldv(int r, IX i, IX sb) const
    {
        return ld_val(r < N_GEO ? v + go(r, i) : shv + so(r, sb));
    }
    // v of plane r, or 0 without loading it (momentum SGD keeps no v)
    template <int OPT> __device__ __forceinline__ float ldv_opt(int r, IX i, IX sb) const
    {
        return OPT == GS_OPT_SGDM ? 0.f : ldv(r, i, sb);
    }
    // Store the updated w, m, v of plane r (rounded per the storage; `key` is
    // sr_plane_key of this plane and step) and, for a geometry plane, the
    // restore direction of what was stored.
    template <int OPT>
    __device__ __forceinline__ void store(int r, IX i, IX sb, float w, float mm, float vv, const SLut &L,
                                          uint32_t key) const
    {
        const bool st = L.stochastic != 0, sgd = OPT == GS_OPT_SGDM;
        const uint32_t bits = st ? sr_bits(key, (uint32_t)i) : 0u;
        if (r < N_GEO) {
            const IX o = go(r, i);
            const float ms = st_val(m + o, mm, st, bits);
            const float vs = sgd ? 0.f : st_val(v + o, vv, st, bits >> 16);
            geo[o] = w;
            if (rdir) rdir[o] = restore_dir<OPT>(ms, vs, L.eps);
        } else {
            const IX o = so(r, sb);
            const float ms = st_val(shm + o, mm, st, bits);
            const float vs = sgd ? 0.f : st_val(shv + o, vv, st, bits >> 16);
            (void)ms;
            (void)vs;
            st_val(shw + o, w, st, sr_w_bits(bits));
        }
    }
};

template <typename T, int OPT>
__device__ __forceinline__ void adam_rows(const Planes<T> &P, int D, int64_t i, int k, const float *__restrict__ grad,
                                          int64_t gcap, int d, const SLut &L)
{
    constexpr int UNROLL = 4;
    const int64_t sb = P.shbase(i);
    for (int r0 = 0; r0 < D; r0 += UNROLL) {
        float w_[UNROLL], m_[UNROLL], v_[UNROLL], g_[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
            int r = r0 + u;
            if (r < D) {
                w_[u] = P.ldw(r, i, sb);
                m_[u] = P.ldm(r, i, sb);
                v_[u] = P.template ldv_opt<OPT>(r, i, sb);
                g_[u] = k >= 0 ? __ldg(grad + r * gcap + k) : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
            int r = r0 + u;
            if (r < D) {
                adam_value<OPT>(w_[u], m_[u], v_[u], g_[u], d, lr_group(r), L);
                P.template store<OPT>(r, i, sb, w_[u], m_[u], v_[u], L,
                                      L.stochastic ? sr_plane_key(L.seed, L.step, (uint32_t)r) : 0u);
            }
        }
    }
}

// One thread per (update-set member, group of RG planes), blockIdx.y selects
// the plane group.  The loads of a thread's next member are issued before the
// current member's arithmetic, so every warp keeps memory requests in flight
// while it computes.  The member's delay comes from the compaction (which
// already cleared its counter).
constexpr int RG = 4;

template <typename IX> struct AdamRows {
    float w[RG], m[RG], v[RG], g[RG];
    IX i, sb;
    int d;
};

template <int OPT, typename T, typename IX>
__device__ __forceinline__ void adam_fetch(AdamRows<IX> &a, int u, const int32_t *__restrict__ uids,
                                           const uint8_t *__restrict__ udelay, const uint32_t *__restrict__ vmask,
                                           const uint32_t *__restrict__ vprefix, const Planes<T, IX> &P,
                                           const float *__restrict__ grad, int64_t gcap, int D, int r0)
{
    a.i = (IX)uids[u];
    a.sb = P.shbase(a.i);
    a.d = udelay[u];
    int k = compact_index(vmask, vprefix, a.i);
    if (k >= gcap) k = -1;     // outside the caller's gradient buffer: treated as zero gradient
#pragma unroll
    for (int j = 0; j < RG; j++) {
        const int r = r0 + j;
        if (r < D) {
            a.w[j] = P.ldw(r, a.i, a.sb);
            a.m[j] = P.ldm(r, a.i, a.sb);
            a.v[j] = P.template ldv_opt<OPT>(r, a.i, a.sb);
            a.g[j] = k >= 0 ? __ldg(grad + r * gcap + k) : 0.f;
        }
    }
}

template <typename T, typename IX, int OPT>
__global__ void __launch_bounds__(ADAM_BLOCK, 4) k_adam_apply(Planes<T, IX> P, int D, const int32_t *__restrict__ uids,
                                                           const uint8_t *__restrict__ udelay, const int *u_range,
                                                           const int *n_upd_p,
                                                           const uint32_t *__restrict__ vmask,
                                                           const uint32_t *__restrict__ vprefix,
                                                           const float *__restrict__ grad, int64_t gcap,
                                                           const DevArgs *__restrict__ args)
{
    __shared__ SLut L;
    load_slut(L, args->lut);
    // members [u_range[0], u_range[1]) of the update set, or all of them
    const int n_upd = u_range ? u_range[1] : *n_upd_p;
    const int r0 = blockIdx.y * RG;
    const int stride = gridDim.x * blockDim.x;
    int u = (u_range ? u_range[0] : 0) + blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_upd) return;
    uint32_t key[RG];          // stochastic-rounding keys of this thread's planes
#pragma unroll
    for (int j = 0; j < RG; j++) key[j] = L.stochastic ? sr_plane_key(L.seed, L.step, (uint32_t)(r0 + j)) : 0u;
    AdamRows<IX> cur, nxt;
    adam_fetch<OPT>(cur, u, uids, udelay, vmask, vprefix, P, grad, gcap, D, r0);
    while (true) {
        const int un = u + stride;
        const bool more = un < n_upd;
        if (more) adam_fetch<OPT>(nxt, un, uids, udelay, vmask, vprefix, P, grad, gcap, D, r0);
#pragma unroll
        for (int j = 0; j < RG; j++) {
            const int r = r0 + j;
            if (r < D) {
                float w_ = cur.w[j], m_ = cur.m[j], v_ = cur.v[j];
                adam_value<OPT>(w_, m_, v_, cur.g[j], cur.d, lr_group(r), L);
                P.template store<OPT>(r, cur.i, cur.sb, w_, m_, v_, L, key[j]);
            }
        }
        if (!more) break;
        cur = nxt;
        u = un;
    }
}

template <typename T, typename IX = int64_t> static Planes<T, IX> planes_of(const SceneView &sc)
{
    Planes<T, IX> P;
    P.geo = sc.geo;
    P.m = (T *)sc.m;
    P.v = (T *)sc.v;
    P.rdir = sc.rdir;
    P.shw = (T *)sc.sh.w;
    P.shm = (T *)sc.sh.m;
    P.shv = (T *)sc.sh.v;
    P.pitch = (IX)sc.pitch;
    P.sp = (IX)sc.sh.ppitch;
    P.slot = sc.sh.slot;
    P.shift = sc.sh.shift;
    return P;
}

// 32-bit element offsets when every plane offset fits (D * pitch and the
// staging ring below 2^32): one multiply-add per address instead of 64-bit math.
static bool offsets_fit_u32(const SceneView &sc)
{
    const uint64_t lim = 1ull << 32;
    return (uint64_t)sc.D * (uint64_t)sc.pitch < lim && (uint64_t)(sc.D - N_GEO) * (uint64_t)sc.sh.ppitch < lim;
}

void launch_adam_select(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, uint32_t *umask,
                        uint32_t *uchunk, int32_t *uids, uint8_t *udelay, int *n_upd, Work &w, cudaStream_t s)
{
    int64_t nchunks = (sc.n + CHUNK - 1) / CHUNK;
    k_adam_select<<<w.grid(nchunks * ADAM_BLOCK, ADAM_BLOCK), ADAM_BLOCK, 0, s>>>(sc.counter, vmask, sc.n, args, umask,
                                                                                uchunk);
    compact_mask(umask, sc.n, uchunk, true, uids, nullptr, (int)sc.n, n_upd, w, s, sc.counter, udelay);
}

// The update-set compaction alone (when the select ran inside the cull sweep).
void launch_adam_compact(const SceneView &sc, uint32_t *umask, uint32_t *uchunk, int32_t *uids, uint8_t *udelay,
                         int *n_upd, Work &w, cudaStream_t s)
{
    compact_mask(umask, sc.n, uchunk, true, uids, nullptr, (int)sc.n, n_upd, w, s, sc.counter, udelay);
}

// Host tier: chunk touch map from the step's masks -- 2 = a Gaussian visible in
// some view, 1 = only update-set members (counter at the bound), else 0.
__global__ void __launch_bounds__(ADAM_BLOCK) k_touch_from_masks(const uint32_t *__restrict__ vmask,
                                                                 const uint32_t *__restrict__ umask, int64_t n,
                                                                 int shift, uint8_t *__restrict__ touch)
{
    const int64_t R = 1ll << shift, nchunks = (n + R - 1) >> shift;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t w0 = (c << shift) >> 5, w1 = (min(n, (c + 1) << shift) + 31) >> 5;
        int vis = 0, upd = 0;
        for (int64_t wd = w0 + threadIdx.x; wd < w1; wd += blockDim.x) {
            vis |= vmask[wd] != 0u;
            upd |= umask[wd] != 0u;
        }
        vis = __syncthreads_or(vis);
        upd = __syncthreads_or(upd);
        if (threadIdx.x == 0) touch[c] = vis ? 2 : (upd ? 1 : 0);
    }
}

void launch_touch_from_masks(const uint32_t *vmask, const uint32_t *umask, int64_t n, int shift, uint8_t *touch,
                             Work &w, cudaStream_t s)
{
    const int64_t nchunks = (n + (1ll << shift) - 1) >> shift;
    k_touch_from_masks<<<w.grid(nchunks * ADAM_BLOCK, ADAM_BLOCK, 4), ADAM_BLOCK, 0, s>>>(vmask, umask, n, shift,
                                                                                       touch);
}

void launch_adam_apply(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                       const float *grad, int64_t gcap, const int32_t *uids, const uint8_t *udelay,
                       const int *u_range, const int *n_upd, Work &w, cudaStream_t s)
{
    const int groups = (sc.D + RG - 1) / RG;
    dim3 grid(w.grid(sc.n, ADAM_BLOCK, 32) / groups + 1, groups);
    const bool u32 = offsets_fit_u32(sc);
    with_opt(sc.opt, [&](auto o) {
        constexpr int O = decltype(o)::value;
        if (sc.prec == GS_FP32) {
            if (u32)
                k_adam_apply<float, uint32_t, O><<<grid, ADAM_BLOCK, 0, s>>>(
                    planes_of<float, uint32_t>(sc), sc.D, uids, udelay, u_range, n_upd, vmask, vprefix, grad, gcap, args);
            else
                k_adam_apply<float, int64_t, O><<<grid, ADAM_BLOCK, 0, s>>>(
                    planes_of<float, int64_t>(sc), sc.D, uids, udelay, u_range, n_upd, vmask, vprefix, grad, gcap, args);
        } else {
            if (u32)
                k_adam_apply<__nv_bfloat16, uint32_t, O><<<grid, ADAM_BLOCK, 0, s>>>(
                    planes_of<__nv_bfloat16, uint32_t>(sc), sc.D, uids, udelay, u_range, n_upd, vmask, vprefix, grad,
                    gcap, args);
            else
                k_adam_apply<__nv_bfloat16, int64_t, O><<<grid, ADAM_BLOCK, 0, s>>>(
                    planes_of<__nv_bfloat16, int64_t>(sc), sc.D, uids, udelay, u_range, n_upd, vmask, vprefix, grad,
                    gcap, args);
        }
    });
}

void launch_adam_deferred(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                          const float *grad, int64_t gcap, uint32_t *umask, uint32_t *uchunk, int32_t *uids,
                          uint8_t *udelay, int *n_upd, Work &w, cudaStream_t s, const PairBufs *pb)
{
    if (pb && adam_pairs_ok(sc)) {
        int64_t nchunks = (sc.n + CHUNK - 1) / CHUNK;
        k_adam_select<<<w.grid(nchunks * ADAM_BLOCK, ADAM_BLOCK), ADAM_BLOCK, 0, s>>>(sc.counter, vmask, sc.n, args,
                                                                                    umask, uchunk);
        launch_adam_pairs(sc, args, vmask, vprefix, grad, gcap, umask, uchunk, *pb, n_upd, w, s);
        return;
    }
    launch_adam_select(sc, args, vmask, umask, uchunk, uids, udelay, n_upd, w, s);
    w.mark(TP_APPLY0, s);
    launch_adam_apply(sc, args, vmask, vprefix, grad, gcap, uids, udelay, nullptr, n_upd, w, s);
    w.mark(TP_APPLY1, s);
}

// ---------------------------------------------------------------------------
// The apply over Gaussian pairs (resident scenes).  The update set is taken as
// pairs (2p, 2p + 1) with at least one member: a thread moves both Gaussians of
// a pair with one 8-byte (fp32) or 4-byte (bf16) access per array and plane,
// twice the bytes per instruction of the member-wise apply (Morton order keeps
// most members in runs, so most pairs are whole).  Each block handles one
// group of PR planes that are all geometry planes or all SH planes, so the
// per-plane code has no branch on the plane's kind.  The arithmetic of each
// member is the member-wise apply's, operation for operation (same results);
// a non-member of a pair is not written.

// Pair mask from the update-set mask: bit p of word w is bit 2p | bit 2p + 1.
__device__ __forceinline__ uint32_t pair_bits16(uint32_t u)
{
    uint32_t x = (u | (u >> 1)) & 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0f0f0f0fu;
    x = (x | (x >> 4)) & 0x00ff00ffu;
    return (x | (x >> 8)) & 0x0000ffffu;
}

__global__ void k_pair_mask(const uint32_t *__restrict__ umask, int64_t nwords_u, uint32_t *__restrict__ pmask,
                            int64_t nwords_p)
{
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords_p; w += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t u0 = 2 * w < nwords_u ? umask[2 * w] : 0u, u1 = 2 * w + 1 < nwords_u ? umask[2 * w + 1] : 0u;
        pmask[w] = pair_bits16(u0) | (pair_bits16(u1) << 16);
    }
}

// Per active pair: both delays and the member bits (d0 | d1 << 8 | members << 16);
// with `clear`, the members' counters are cleared (the compaction's job in the
// member path), else the apply clears them.
__global__ void k_pair_prep(const int32_t *__restrict__ pids, const int *n_pairs_p, const uint32_t *__restrict__ umask,
                            uint8_t *__restrict__ counter, int64_t n, uint32_t *__restrict__ pinfo, int clear)
{
    const int np = *n_pairs_p;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += gridDim.x * blockDim.x) {
        const int64_t i0 = 2 * (int64_t)pids[j];
        const bool has1 = i0 + 1 < n;
        uint32_t bits = (umask[i0 >> 5] >> (i0 & 31)) & (has1 ? 3u : 1u);
        const uint32_t c0 = counter[i0], c1 = has1 ? counter[i0 + 1] : 0u;
        if (clear && (bits & 1u)) counter[i0] = 0;
        if (clear && (bits & 2u)) counter[i0 + 1] = 0;
        pinfo[j] = c0 | (c1 << 8) | (bits << 16);
    }
}

// Two consecutive elements of a plane: loads widen to fp32, stores round per
// the storage (stochastically with the member-wise apply's bits for bf16).
__device__ __forceinline__ void ld2(const float *p, float &a, float &b)
{
    const float2 v = *reinterpret_cast<const float2 *>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld2(const __nv_bfloat16 *p, float &a, float &b)
{
    const uint32_t u = *reinterpret_cast<const uint32_t *>(p);
    a = __uint_as_float(u << 16);
    b = __uint_as_float(u & 0xffff0000u);
}

// Rounded representation of x in T: returns the bits and the value as stored.
__device__ __forceinline__ uint32_t rnd_bits(float x, float &stored, const float *, bool, uint32_t)
{
    stored = x;
    return __float_as_uint(x);
}
__device__ __forceinline__ uint32_t rnd_bits(float x, float &stored, const __nv_bfloat16 *, bool stochastic, uint32_t rnd)
{
    uint32_t u = __float_as_uint(x);
    uint16_t b;
    if (!stochastic || (u & 0x7f800000u) == 0x7f800000u) {
        b = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    } else {
        u += rnd & 0xffffu;
        b = (uint16_t)(u >> 16);
    }
    stored = __uint_as_float((uint32_t)b << 16);
    return b;
}

// Store the pair's elements whose bit is set in `sel` (bits a, b as from rnd_bits).
__device__ __forceinline__ void st2(float *p, uint32_t a, uint32_t b, uint32_t sel)
{
    if (sel == 3u) *reinterpret_cast<float2 *>(p) = make_float2(__uint_as_float(a), __uint_as_float(b));
    else if (sel == 1u) p[0] = __uint_as_float(a);
    else if (sel == 2u) p[1] = __uint_as_float(b);
}
__device__ __forceinline__ void st2(__nv_bfloat16 *p, uint32_t a, uint32_t b, uint32_t sel)
{
    if (sel == 3u) *reinterpret_cast<uint32_t *>(p) = a | (b << 16);
    else if (sel == 1u) p[0] = __ushort_as_bfloat16((unsigned short)a);
    else if (sel == 2u) p[1] = __ushort_as_bfloat16((unsigned short)b);
}

constexpr int PR = 2;      // planes per thread in the pair apply

struct PairRows {
    float w[PR][2], m[PR][2], v[PR][2], g[PR][2];
    int64_t i0;
    uint32_t info;
};

// Planes [r0, r0 + PR) of one kind: geometry (w fp32 at geo, m, v of type T,
// directions fp32) or SH (all of type T).
template <typename T, bool GEO, int OPT>
__device__ __forceinline__ void pair_fetch(PairRows &a, int j, const int32_t *__restrict__ pids,
                                           const uint32_t *__restrict__ pinfo, const Planes<T> &P,
                                           const uint32_t *__restrict__ vmask, const uint32_t *__restrict__ vprefix,
                                           const float *__restrict__ grad, int64_t gcap, int r0, int rend)
{
    a.i0 = 2 * (int64_t)pids[j];
    a.info = pinfo[j];
    int k0 = (a.info & (1u << 16)) ? compact_index(vmask, vprefix, a.i0) : -1;
    int k1 = (a.info & (2u << 16)) ? compact_index(vmask, vprefix, a.i0 + 1) : -1;
    if (k0 >= gcap) k0 = -1;
    if (k1 >= gcap) k1 = -1;
#pragma unroll
    for (int q = 0; q < PR; q++) {
        const int r = r0 + q;
        if (r < rend) {
            if (GEO) {
                ld2(P.geo + (int64_t)r * P.pitch + a.i0, a.w[q][0], a.w[q][1]);
                ld2(P.m + (int64_t)r * P.pitch + a.i0, a.m[q][0], a.m[q][1]);
                if (OPT != GS_OPT_SGDM) ld2(P.v + (int64_t)r * P.pitch + a.i0, a.v[q][0], a.v[q][1]);
            } else {
                const int64_t o = (int64_t)(r - N_GEO) * P.sp + a.i0;
                ld2(P.shw + o, a.w[q][0], a.w[q][1]);
                ld2(P.shm + o, a.m[q][0], a.m[q][1]);
                if (OPT != GS_OPT_SGDM) ld2(P.shv + o, a.v[q][0], a.v[q][1]);
            }
            if (OPT == GS_OPT_SGDM) a.v[q][0] = a.v[q][1] = 0.f;
            a.g[q][0] = k0 >= 0 ? __ldg(grad + (int64_t)r * gcap + k0) : 0.f;
            a.g[q][1] = k1 >= 0 ? __ldg(grad + (int64_t)r * gcap + k1) : 0.f;
        }
    }
}

template <typename T, bool GEO, int OPT>
__device__ __forceinline__ void pair_step(const PairRows &a, const Planes<T> &P, int r0, int rend, const SLut &L,
                                          const uint32_t *key)
{
    const uint32_t sel = (a.info >> 16) & 3u;
    const int dd[2] = {(int)(a.info & 255u), (int)((a.info >> 8) & 255u)};
    const bool st = L.stochastic != 0;
#pragma unroll
    for (int q = 0; q < PR; q++) {
        const int r = r0 + q;
        if (r >= rend) continue;
        const int grp = lr_group(r);
        uint32_t bw[2], bm[2], bv[2], bd[2];
#pragma unroll
        for (int e = 0; e < 2; e++) {
            float w = a.w[q][e], m = a.m[q][e], v = a.v[q][e];
            bw[e] = bm[e] = bv[e] = bd[e] = 0u;
            if (!((sel >> e) & 1u)) continue;
            adam_value<OPT>(w, m, v, a.g[q][e], dd[e], grp, L);
            const uint32_t bits = st ? sr_bits(key[q], (uint32_t)(a.i0 + e)) : 0u;
            float ms, vs, ws;
            if (GEO) {
                bm[e] = rnd_bits(m, ms, P.m, st, bits);
                bv[e] = OPT == GS_OPT_SGDM ? 0u : rnd_bits(v, vs, P.v, st, bits >> 16);
                bw[e] = __float_as_uint(w);
                bd[e] = __float_as_uint(restore_dir<OPT>(ms, OPT == GS_OPT_SGDM ? 0.f : vs, L.eps));
            } else {
                bm[e] = rnd_bits(m, ms, P.shm, st, bits);
                bv[e] = OPT == GS_OPT_SGDM ? 0u : rnd_bits(v, vs, P.shv, st, bits >> 16);
                bw[e] = rnd_bits(w, ws, P.shw, st, sr_w_bits(bits));
            }
        }
        if (GEO) {
            const int64_t o = (int64_t)r * P.pitch + a.i0;
            st2(P.geo + o, bw[0], bw[1], sel);
            st2(P.m + o, bm[0], bm[1], sel);
            if (OPT != GS_OPT_SGDM) st2(P.v + o, bv[0], bv[1], sel);
            if (P.rdir) st2(P.rdir + o, bd[0], bd[1], sel);
        } else {
            const int64_t o = (int64_t)(r - N_GEO) * P.sp + a.i0;
            st2(P.shw + o, bw[0], bw[1], sel);
            st2(P.shm + o, bm[0], bm[1], sel);
            if (OPT != GS_OPT_SGDM) st2(P.shv + o, bv[0], bv[1], sel);
        }
    }
}

// bf16 form: both elements of a pair rounded by one conversion instruction
// (cvt.rn / cvt.rs .bf16x2.f32; element 0 in the low half).  Stochastic
// rounding (cvt.rs) takes 16 random bits per element from rbits, the low half
// for element 0: the same bits the per-element path adds below the kept
// mantissa (sr_bits of each element, low 16 bits for m, high 16 for v,
// sr_w_bits for w).
__device__ __forceinline__ uint32_t bf16x2_round(float x0, float x1, bool stochastic, uint32_t rbits)
{
    uint32_t d;
    if (stochastic)
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(x1), "f"(x0), "r"(rbits));
    else
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(x1), "f"(x0));
    return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t d) { return __uint_as_float(d << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t d) { return __uint_as_float(d & 0xffff0000u); }

// Store the halves of a packed bf16 pair whose bit is set in `sel`.
__device__ __forceinline__ void st2p(__nv_bfloat16 *p, uint32_t d, uint32_t sel)
{
    if (sel == 3u) *reinterpret_cast<uint32_t *>(p) = d;
    else if (sel == 1u) reinterpret_cast<uint16_t *>(p)[0] = (uint16_t)d;
    else if (sel == 2u) reinterpret_cast<uint16_t *>(p)[1] = (uint16_t)(d >> 16);
}

template <bool GEO, int OPT>
__device__ __forceinline__ void pair_step_bf16(const PairRows &a, const Planes<__nv_bfloat16> &P, int r0, int rend,
                                               const SLut &L, const uint32_t *key)
{
    const uint32_t sel = (a.info >> 16) & 3u;
    const int dd[2] = {(int)(a.info & 255u), (int)((a.info >> 8) & 255u)};
    const bool st = L.stochastic != 0;
#pragma unroll
    for (int q = 0; q < PR; q++) {
        const int r = r0 + q;
        if (r >= rend) continue;
        const int grp = lr_group(r);
        float w[2], m[2], v[2];
#pragma unroll
        for (int e = 0; e < 2; e++) {
            w[e] = a.w[q][e];
            m[e] = a.m[q][e];
            v[e] = a.v[q][e];
            if ((sel >> e) & 1u) adam_value<OPT>(w[e], m[e], v[e], a.g[q][e], dd[e], grp, L);
        }
        const uint32_t h0 = st ? sr_bits(key[q], (uint32_t)a.i0) : 0u;
        const uint32_t h1 = st ? sr_bits(key[q], (uint32_t)(a.i0 + 1)) : 0u;
        const uint32_t pm = bf16x2_round(m[0], m[1], st, (h0 & 0xffffu) | (h1 << 16));
        const uint32_t pv = OPT == GS_OPT_SGDM ? 0u : bf16x2_round(v[0], v[1], st, (h0 >> 16) | (h1 & 0xffff0000u));
        if (GEO) {
            const int64_t o = (int64_t)r * P.pitch + a.i0;
            st2(P.geo + o, __float_as_uint(w[0]), __float_as_uint(w[1]), sel);
            st2p(P.m + o, pm, sel);
            if (OPT != GS_OPT_SGDM) st2p(P.v + o, pv, sel);
            if (P.rdir) {
                const float d0 = restore_dir<OPT>(bf16_lo(pm), bf16_lo(pv), L.eps);
                const float d1 = restore_dir<OPT>(bf16_hi(pm), bf16_hi(pv), L.eps);
                st2(P.rdir + o, __float_as_uint(d0), __float_as_uint(d1), sel);
            }
        } else {
            const uint32_t pw = bf16x2_round(w[0], w[1], st, (sr_w_bits(h0) & 0xffffu) | (sr_w_bits(h1) << 16));
            const int64_t o = (int64_t)(r - N_GEO) * P.sp + a.i0;
            st2p(P.shw + o, pw, sel);
            st2p(P.shm + o, pm, sel);
            if (OPT != GS_OPT_SGDM) st2p(P.shv + o, pv, sel);
        }
    }
}

// bf16 SH planes: four planes per thread, each array's pair of values kept
// packed (one bf16x2 register) until it is stepped.  The arithmetic of each
// plane is pair_step_bf16's.
constexpr int PR_SH16 = 4;
struct PairRowsSH16 {
    uint32_t w[PR_SH16], m[PR_SH16], v[PR_SH16];
    float g[PR_SH16][2];
    int64_t i0;
    uint32_t info;
};

template <int OPT>
__device__ __forceinline__ void pair_fetch_sh16(PairRowsSH16 &a, int j, const int32_t *__restrict__ pids,
                                                const uint32_t *__restrict__ pinfo,
                                                const Planes<__nv_bfloat16> &P, const uint32_t *__restrict__ vmask,
                                                const uint32_t *__restrict__ vprefix, const float *__restrict__ grad,
                                                int64_t gcap, int r0, int rend)
{
    a.i0 = 2 * (int64_t)pids[j];
    a.info = pinfo[j];
    int k0 = (a.info & (1u << 16)) ? compact_index(vmask, vprefix, a.i0) : -1;
    int k1 = (a.info & (2u << 16)) ? compact_index(vmask, vprefix, a.i0 + 1) : -1;
    if (k0 >= gcap) k0 = -1;
    if (k1 >= gcap) k1 = -1;
#pragma unroll
    for (int q = 0; q < PR_SH16; q++) {
        const int r = r0 + q;
        if (r < rend) {
            const int64_t o = (int64_t)(r - N_GEO) * P.sp + a.i0;
            a.w[q] = *reinterpret_cast<const uint32_t *>(P.shw + o);
            a.m[q] = *reinterpret_cast<const uint32_t *>(P.shm + o);
            a.v[q] = OPT == GS_OPT_SGDM ? 0u : *reinterpret_cast<const uint32_t *>(P.shv + o);
            a.g[q][0] = k0 >= 0 ? __ldg(grad + (int64_t)r * gcap + k0) : 0.f;
            a.g[q][1] = k1 >= 0 ? __ldg(grad + (int64_t)r * gcap + k1) : 0.f;
        }
    }
}

template <int OPT>
__device__ __forceinline__ void pair_step_sh16(const PairRowsSH16 &a, const Planes<__nv_bfloat16> &P, int r0, int rend,
                                               const SLut &L, const uint32_t *key)
{
    const uint32_t sel = (a.info >> 16) & 3u;
    const int dd[2] = {(int)(a.info & 255u), (int)((a.info >> 8) & 255u)};
    const bool st = L.stochastic != 0;
#pragma unroll
    for (int q = 0; q < PR_SH16; q++) {
        const int r = r0 + q;
        if (r >= rend) continue;
        const int grp = lr_group(r);
        float w[2] = {bf16_lo(a.w[q]), bf16_hi(a.w[q])}, m[2] = {bf16_lo(a.m[q]), bf16_hi(a.m[q])};
        float v[2] = {bf16_lo(a.v[q]), bf16_hi(a.v[q])};
#pragma unroll
        for (int e = 0; e < 2; e++)
            if ((sel >> e) & 1u) adam_value<OPT>(w[e], m[e], v[e], a.g[q][e], dd[e], grp, L);
        const uint32_t h0 = st ? sr_bits(key[q], (uint32_t)a.i0) : 0u;
        const uint32_t h1 = st ? sr_bits(key[q], (uint32_t)(a.i0 + 1)) : 0u;
        const uint32_t pm = bf16x2_round(m[0], m[1], st, (h0 & 0xffffu) | (h1 << 16));
        const uint32_t pv = OPT == GS_OPT_SGDM ? 0u : bf16x2_round(v[0], v[1], st, (h0 >> 16) | (h1 & 0xffff0000u));
        const uint32_t pw = bf16x2_round(w[0], w[1], st, (sr_w_bits(h0) & 0xffffu) | (sr_w_bits(h1) << 16));
        const int64_t o = (int64_t)(r - N_GEO) * P.sp + a.i0;
        st2p(P.shw + o, pw, sel);
        st2p(P.shm + o, pm, sel);
        if (OPT != GS_OPT_SGDM) st2p(P.shv + o, pv, sel);
    }
}

template <typename T, bool GEO, int OPT>
__device__ __forceinline__ void pair_step_any(const PairRows &a, const Planes<T> &P, int r0, int rend, const SLut &L,
                                              const uint32_t *key)
{
    if constexpr (std::is_same<T, __nv_bfloat16>::value)
        pair_step_bf16<GEO, OPT>(a, P, r0, rend, L, key);
    else
        pair_step<T, GEO, OPT>(a, P, r0, rend, L, key);
}

// blockIdx.y: plane groups; the first n_geo_groups cover geometry planes
// [PR y, PR y + PR) below 11, the rest SH planes 11 + PS (y - n_geo_groups) ...
// with PS = PR (fp32) or PR_SH16 (bf16).
template <typename T> __host__ __device__ constexpr int sh_planes_per_thread() { return std::is_same<T, __nv_bfloat16>::value ? PR_SH16 : PR; }

template <typename T, int OPT>
__global__ void __launch_bounds__(ADAM_BLOCK, 4) k_adam_apply_pairs(Planes<T> P, int D, const int32_t *__restrict__ pids,
                                                                 const uint32_t *__restrict__ pinfo,
                                                                 const int *n_pairs_p,
                                                                 const uint32_t *__restrict__ vmask,
                                                                 const uint32_t *__restrict__ vprefix,
                                                                 const float *__restrict__ grad, int64_t gcap,
                                                                 const DevArgs *__restrict__ args,
                                                                 uint8_t *__restrict__ counter_clear)
{
    __shared__ SLut L;
    load_slut(L, args->lut);
    const int n_pairs = *n_pairs_p;
    constexpr int GEO_GROUPS = (N_GEO + PR - 1) / PR;
    constexpr int PS = sh_planes_per_thread<T>();
    const bool geo = blockIdx.y < GEO_GROUPS;
    const int r0 = geo ? (int)blockIdx.y * PR : N_GEO + ((int)blockIdx.y - GEO_GROUPS) * PS;
    const int rend = geo ? N_GEO : D;
    const int stride = gridDim.x * blockDim.x;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pairs) return;
    uint32_t key[PS];
#pragma unroll
    for (int q = 0; q < PS; q++) key[q] = L.stochastic ? sr_plane_key(L.seed, L.step, (uint32_t)(r0 + q)) : 0u;
    if constexpr (PS == PR_SH16) {
        if (!geo) {
            // four planes' loads in flight per pair (as many as the fp32 form's two planes of this pair
            // and the next): no prefetch of the next pair
            for (; j < n_pairs; j += stride) {
                PairRowsSH16 c16;
                pair_fetch_sh16<OPT>(c16, j, pids, pinfo, P, vmask, vprefix, grad, gcap, r0, rend);
                pair_step_sh16<OPT>(c16, P, r0, rend, L, key);
            }
            return;
        }
    }
    PairRows cur, nxt;
    // the first plane group clears the members' counters (when the pair
    // preparation left them)
    uint8_t *const clr = blockIdx.y == 0 ? counter_clear : nullptr;
    if (geo) {
        pair_fetch<T, true, OPT>(cur, j, pids, pinfo, P, vmask, vprefix, grad, gcap, r0, rend);
        while (true) {
            const int jn = j + stride;
            const bool more = jn < n_pairs;
            if (more) pair_fetch<T, true, OPT>(nxt, jn, pids, pinfo, P, vmask, vprefix, grad, gcap, r0, rend);
            pair_step_any<T, true, OPT>(cur, P, r0, rend, L, key);
            if (clr) {
                if (cur.info & (1u << 16)) clr[cur.i0] = 0;
                if (cur.info & (2u << 16)) clr[cur.i0 + 1] = 0;
            }
            if (!more) break;
            cur = nxt;
            j = jn;
        }
    } else {
        pair_fetch<T, false, OPT>(cur, j, pids, pinfo, P, vmask, vprefix, grad, gcap, r0, rend);
        while (true) {
            const int jn = j + stride;
            const bool more = jn < n_pairs;
            if (more) pair_fetch<T, false, OPT>(nxt, jn, pids, pinfo, P, vmask, vprefix, grad, gcap, r0, rend);
            pair_step_any<T, false, OPT>(cur, P, r0, rend, L, key);
            if (!more) break;
            cur = nxt;
            j = jn;
        }
    }
}

bool adam_pairs_ok(const SceneView &sc)
{
    // resident planes, 8-byte aligned pair accesses (pitch is a multiple of 4)
    auto al = [](const void *p) { return ((uintptr_t)p & 7) == 0; };
    return !sc.sh.slot && al(sc.geo) && al(sc.m) && al(sc.v) && al(sc.sh.w) && al(sc.sh.m) && al(sc.sh.v) &&
           (!sc.rdir || al(sc.rdir)) && sc.counter;
}

static void pairs_prep(const SceneView &sc, uint32_t *umask, uint32_t *uchunk, const PairBufs &pb, int *n_upd,
                       bool clear, Work &w, cudaStream_t s)
{
    const int64_t nw_u = (sc.n + 31) / 32, npairs = (sc.n + 1) / 2, nw_p = (npairs + 31) / 32;
    // members of the update set (reported), from the per-chunk counts of the select
    scan_counts(uchunk, (sc.n + CHUNK - 1) / CHUNK, n_upd, 0, w, s);
    k_pair_mask<<<w.grid(nw_p, 256, 4), 256, 0, s>>>(umask, nw_u, pb.pmask, nw_p);
    compact_mask(pb.pmask, npairs, pb.pchunk, false, pb.pids, nullptr, (int)npairs, pb.n_pairs, w, s);
    k_pair_prep<<<w.grid(npairs, 256, 4), 256, 0, s>>>(pb.pids, pb.n_pairs, umask, sc.counter, sc.n, pb.pinfo,
                                                       clear ? 1 : 0);
}

static void pairs_apply(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                        const float *grad, int64_t gcap, const PairBufs &pb, uint8_t *counter_clear, Work &w,
                        cudaStream_t s)
{
    constexpr int GEO_GROUPS = (N_GEO + PR - 1) / PR;
    const int ps = sc.prec == GS_FP32 ? sh_planes_per_thread<float>() : sh_planes_per_thread<__nv_bfloat16>();
    const int groups = GEO_GROUPS + (sc.D - N_GEO + ps - 1) / ps;
    dim3 grid(w.grid(sc.n, ADAM_BLOCK, 32) / groups + 1, groups);
    w.mark(TP_APPLY0, s);
    with_opt(sc.opt, [&](auto o) {
        constexpr int O = decltype(o)::value;
        if (sc.prec == GS_FP32)
            k_adam_apply_pairs<float, O><<<grid, ADAM_BLOCK, 0, s>>>(planes_of<float>(sc), sc.D, pb.pids, pb.pinfo,
                                                                    pb.n_pairs, vmask, vprefix, grad, gcap, args,
                                                                    counter_clear);
        else
            k_adam_apply_pairs<__nv_bfloat16, O><<<grid, ADAM_BLOCK, 0, s>>>(
                planes_of<__nv_bfloat16>(sc), sc.D, pb.pids, pb.pinfo, pb.n_pairs, vmask, vprefix, grad, gcap, args,
                counter_clear);
    });
    w.mark(TP_APPLY1, s);
}

void launch_adam_pairs(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                       const float *grad, int64_t gcap, uint32_t *umask, uint32_t *uchunk, const PairBufs &pb,
                       int *n_upd, Work &w, cudaStream_t s)
{
    pairs_prep(sc, umask, uchunk, pb, n_upd, true, w, s);
    pairs_apply(sc, args, vmask, vprefix, grad, gcap, pb, nullptr, w, s);
}

void launch_adam_pairs_prep(const SceneView &sc, uint32_t *umask, uint32_t *uchunk, const PairBufs &pb, int *n_upd,
                            Work &w, cudaStream_t s)
{
    // scans on their own partials: this may run beside the main stream's scans
    Work ws = w;
    ws.partials = w.partials + 1024;
    pairs_prep(sc, umask, uchunk, pb, n_upd, false, ws, s);
}

void launch_adam_pairs_apply(const SceneView &sc, const DevArgs *args, const uint32_t *vmask,
                             const uint32_t *vprefix, const float *grad, int64_t gcap, const PairBufs &pb, Work &w,
                             cudaStream_t s)
{
    pairs_apply(sc, args, vmask, vprefix, grad, gcap, pb, sc.counter, w, s);
}

// [first, end) of the update-set members with ids in [id_lo, id_hi): the ids
// are ascending, so two binary searches.
__global__ void k_uid_range(const int32_t *__restrict__ uids, const int *n_upd_p, int64_t id_lo, int64_t id_hi,
                            int *range)
{
    if (threadIdx.x >= 2) return;
    const int64_t key = threadIdx.x == 0 ? id_lo : id_hi;
    int lo = 0, hi = *n_upd_p;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (uids[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    range[threadIdx.x] = lo;
}

void launch_uid_range(const int32_t *uids, const int *n_upd, int64_t id_lo, int64_t id_hi, int *range, cudaStream_t s)
{
    k_uid_range<<<1, 32, 0, s>>>(uids, n_upd, id_lo, id_hi, range);
}

// Eager Adam (Eq. 1 for every Gaussian, every step): the baseline the
// deferred update removes; counters are left alone.
template <typename T, int OPT>
__global__ void __launch_bounds__(ADAM_BLOCK) k_adam_eager(Planes<T> P, int64_t n, int D,
                                                           const uint32_t *__restrict__ vmask,
                                                           const uint32_t *__restrict__ vprefix,
                                                           const float *__restrict__ grad, int64_t gcap,
                                                           const DevArgs *__restrict__ args)
{
    __shared__ SLut L;
    load_slut(L, args->lut);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int k = compact_index(vmask, vprefix, i);
        if (k >= gcap) k = -1;
        adam_rows<T, OPT>(P, D, i, k, grad, gcap, 0, L);
    }
}

void launch_adam_eager(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                       const float *grad, int64_t gcap, Work &w, cudaStream_t s)
{
    w.mark(TP_APPLY0, s);
    with_opt(sc.opt, [&](auto o) {
        constexpr int O = decltype(o)::value;
        if (sc.prec == GS_FP32)
            k_adam_eager<float, O><<<w.grid(sc.n, ADAM_BLOCK), ADAM_BLOCK, 0, s>>>(planes_of<float>(sc), sc.n, sc.D,
                                                                                 vmask, vprefix, grad, gcap, args);
        else
            k_adam_eager<__nv_bfloat16, O><<<w.grid(sc.n, ADAM_BLOCK), ADAM_BLOCK, 0, s>>>(
                planes_of<__nv_bfloat16>(sc), sc.n, sc.D, vmask, vprefix, grad, gcap, args);
    });
    w.mark(TP_APPLY1, s);
}

// rdir = m / (sqrt(v) + eps) for every geometry plane (momentum SGD: rdir = m).
template <typename T, int OPT>
__global__ void k_refresh_rdir(Planes<T> P, int64_t n, const DevArgs *__restrict__ args)
{
    const float eps = args->lut.eps;
    const int64_t total = (int64_t)N_GEO * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n);
        const int64_t i = e - (int64_t)r * n;
        P.rdir[r * P.pitch + i] = restore_dir<OPT>(P.ldm(r, i, i), P.template ldv_opt<OPT>(r, i, i), eps);
    }
}

void launch_refresh_rdir(const SceneView &sc, const DevArgs *args, Work &w, cudaStream_t s)
{
    if (!sc.rdir) return;
    const int g = w.grid((int64_t)N_GEO * sc.n, 256, 4);
    with_opt(sc.opt, [&](auto o) {
        constexpr int O = decltype(o)::value;
        if (sc.prec == GS_FP32)
            k_refresh_rdir<float, O><<<g, 256, 0, s>>>(planes_of<float>(sc), sc.n, args);
        else
            k_refresh_rdir<__nv_bfloat16, O><<<g, 256, 0, s>>>(planes_of<__nv_bfloat16>(sc), sc.n, args);
    });
}

// Catch-up without a step: m b1^c, v b2^c, decay[c] w - param_lut[c] m / (sqrt(v) + eps)
// (momentum SGD: b mu^c, v unchanged, w - param_lut[c] b).
template <typename T, int OPT>
__global__ void k_materialize(Planes<T> P, const uint8_t *__restrict__ counter, int64_t n, int D,
                              const DevArgs *__restrict__ args, float *w_out, float *m_out, float *v_out)
{
    __shared__ SLut L;
    load_slut(L, args->lut);
    const int64_t pitch = P.pitch;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int d = counter ? counter[i] : 0;
        const int64_t sb = P.shbase(i);
        for (int r = 0; r < D; r++) {
            float w = P.ldw(r, i, sb);
            float mm = P.ldm(r, i, sb), vv = P.ldv(r, i, sb);
            const int g = lr_group(r);
            if (w_out) w_out[r * pitch + i] = restore_param<OPT>(w, mm, vv, L.param[g][d], L.decay[g][d], d, L.eps);
            if (m_out) m_out[r * pitch + i] = d ? L.mom[d - 1] * mm : mm;
            if (v_out) v_out[r * pitch + i] = d ? L.var[d - 1] * vv : vv;
        }
    }
}

void launch_materialize(const SceneView &sc, const DevArgs *args, float *w_out, float *m_out, float *v_out,
                        Work &w, cudaStream_t s)
{
    with_opt(sc.opt, [&](auto o) {
        constexpr int O = decltype(o)::value;
        if (sc.prec == GS_FP32)
            k_materialize<float, O><<<w.grid(sc.n, 256), 256, 0, s>>>(planes_of<float>(sc), sc.counter, sc.n, sc.D, args,
                                                                    w_out, m_out, v_out);
        else
            k_materialize<__nv_bfloat16, O><<<w.grid(sc.n, 256), 256, 0, s>>>(planes_of<__nv_bfloat16>(sc), sc.counter,
                                                                             sc.n, sc.D, args, w_out, m_out, v_out);
    });
}

__global__ void k_grad_scatter(const int32_t *__restrict__ ids, const int *n_dev, int cap,
                               const float *__restrict__ gc, int64_t gcap, int D, float *gfull, int64_t pitch)
{
    int cnt = min(*n_dev, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        int64_t i = ids[k];
        if (i < 0 || i >= pitch) continue;
        for (int r = 0; r < D; r++) gfull[r * pitch + i] = gc[r * gcap + k];
    }
}

void launch_grad_scatter(const int32_t *ids, const int *n_dev, int cap, const float *gc, int64_t gcap, int D,
                         float *gfull, int64_t pitch, Work &w, cudaStream_t s)
{
    cudaMemsetAsync(gfull, 0, (size_t)D * pitch * sizeof(float), s);
    k_grad_scatter<<<w.grid(cap, 256), 256, 0, s>>>(ids, n_dev, cap, gc, gcap, D, gfull, pitch);
}

}  // namespace gs
