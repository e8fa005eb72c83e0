// k_densify.cu -- densification on deferred optimizer state (§2.4 step 7,
// with the deferred update of §4.3): clone, split and prune of a resident
// scene into a new scene.  The paper names the step and leaves its rules to
// 3DGS: g = accumulated view-space gradient norm / views seen; g >= threshold
// clones a Gaussian whose largest scale is at most percent_dense * extent and
// splits a larger one into two children (scales / 1.6, means mu + R(q) (s z)
// with standard-normal z given by the caller); then a Gaussian whose opacity
// is below min_opacity is pruned.  New Gaussians start with zero moments.
//
// Deferred state: every decision reads current (caught-up) values; a row that
// is cloned or split is caught up first (counter 0); every other row keeps its
// stored values, restore directions and counter.  The opacity of a clone or a
// child is its parent's, so one decision prunes a row together with its
// copies.  Output order: the surviving rows, then the clones, then the first
// children of the splits, then the second children.
//
//   k_densify_classify  one thread per Gaussian: the three masks (survivor,
//                       clone, split) by warp ballots
//   compact_mask        each mask's word prefix and count (k_scan.cu)
//   k_densify_write     one thread per Gaussian: its rows in the new scene
#include "gs_kernels.cuh"

namespace gs {

namespace {

// Plane r of Gaussian i: w (fp32 geometry or T SH), m, v (T), restore direction
// (fp32 geometry, T SH) of a resident scene.
template <typename T> struct DPlanes {
    float *geo;
    T *m, *v, *shw, *shm, *shv;
    float *rdir;
    int64_t pitch;
    __device__ __forceinline__ float w(int r, int64_t i) const
    {
        return r < N_GEO ? geo[r * pitch + i] : ld_val(shw + (r - N_GEO) * pitch + i);
    }
    __device__ __forceinline__ float mm(int r, int64_t i) const
    {
        return ld_val(r < N_GEO ? m + r * pitch + i : shm + (r - N_GEO) * pitch + i);
    }
    __device__ __forceinline__ float vv(int r, int64_t i) const
    {
        return ld_val(r < N_GEO ? v + r * pitch + i : shv + (r - N_GEO) * pitch + i);
    }
    // stores round to nearest (densification draws no random bits); d_ is the
    // restore direction of a geometry plane
    __device__ __forceinline__ void put(int r, int64_t i, float w_, float m_, float v_, float d_) const
    {
        if (r < N_GEO) {
            geo[r * pitch + i] = w_;
            st_val(m + r * pitch + i, m_, false, 0u);
            st_val(v + r * pitch + i, v_, false, 0u);
            if (rdir) rdir[r * pitch + i] = d_;
        } else {
            const int64_t o = (r - N_GEO) * pitch + i;
            st_val(shw + o, w_, false, 0u);
            st_val(shm + o, m_, false, 0u);
            st_val(shv + o, v_, false, 0u);
        }
    }
};

template <typename T> DPlanes<T> dplanes(const SceneView &sc)
{
    DPlanes<T> P;
    P.geo = sc.geo;
    P.m = (T *)sc.m;
    P.v = (T *)sc.v;
    P.shw = (T *)sc.sh.w;
    P.shm = (T *)sc.sh.m;
    P.shv = (T *)sc.sh.v;
    P.rdir = sc.rdir;
    P.pitch = sc.pitch;
    return P;
}

struct DensifyRule {
    float grad_threshold, scale_limit, min_opacity;   // scale_limit = percent_dense * extent
};

// Current value of plane r of Gaussian i (the catch-up of Eq. 3 with the tables
// of the coming step): geometry planes from the stored direction when the
// scene keeps them, SH planes from m and v.
template <typename T, int OPT>
__device__ __forceinline__ float current(const DPlanes<T> &P, const DevLut &L, int r, int64_t i, int d)
{
    if (!d) return P.w(r, i);
    const int g = lr_group(r);
    const float dir = (P.rdir && r < N_GEO) ? P.rdir[r * P.pitch + i] : restore_dir<OPT>(P.mm(r, i), P.vv(r, i), L.eps);
    return restore_with_dir<OPT>(P.w(r, i), dir, L.param[g][d], L.decay[g][d], d);
}

template <typename T, int OPT>
__global__ void __launch_bounds__(256) k_densify_classify(DPlanes<T> P, const uint8_t *__restrict__ counter, int64_t n,
                                                         const DevArgs *__restrict__ args,
                                                         const float *__restrict__ accum,
                                                         const float *__restrict__ denom, DensifyRule rule,
                                                         uint32_t *surv, uint32_t *clone, uint32_t *split)
{
    const DevLut &L = args->lut;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (n + 31) >> 5;
    for (int64_t wbase = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) << 5; wbase < nw * 32;
         wbase += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = wbase + lane;
        bool s = false, c = false, p = false;
        if (i < n) {
            const int d = counter[i];
            const float l0 = current<T, OPT>(P, L, 3, i, d), l1 = current<T, OPT>(P, L, 4, i, d);
            const float l2 = current<T, OPT>(P, L, 5, i, d), op = current<T, OPT>(P, L, ROW_OPAC, i, d);
            const float den = denom[i];
            const float g = den > 0.f ? accum[i] / den : 0.f;
            const float smax = expf(fmaxf(l0, fmaxf(l1, l2)));
            const bool big = g >= rule.grad_threshold;
            const bool small = smax <= rule.scale_limit;
            const bool keep = 1.f / (1.f + expf(-op)) >= rule.min_opacity;
            c = keep && big && small;
            p = keep && big && !small;
            s = keep && !(big && !small);
        }
        const uint32_t ws = __ballot_sync(0xffffffffu, s), wc = __ballot_sync(0xffffffffu, c),
                       wp = __ballot_sync(0xffffffffu, p);
        if (lane == 0) {
            surv[wbase >> 5] = ws;
            clone[wbase >> 5] = wc;
            split[wbase >> 5] = wp;
        }
    }
}

__device__ __forceinline__ bool bit_at(const uint32_t *mask, int64_t i) { return (mask[i >> 5] >> (i & 31)) & 1u; }
__device__ __forceinline__ int64_t rank_at(const uint32_t *mask, const uint32_t *prefix, int64_t i)
{
    return (int64_t)prefix[i >> 5] + __popc(mask[i >> 5] & ((1u << (i & 31)) - 1u));
}

template <typename T, int OPT>
__global__ void __launch_bounds__(256) k_densify_write(DPlanes<T> P, const uint8_t *__restrict__ counter, int64_t n,
                                                      int D, const DevArgs *__restrict__ args,
                                                      const float *__restrict__ normals, const uint32_t *surv,
                                                      const uint32_t *sprefix, const uint32_t *clone,
                                                      const uint32_t *cprefix, const uint32_t *split,
                                                      const uint32_t *pprefix, const int *counts, DPlanes<T> Q,
                                                      uint8_t *__restrict__ qcounter)
{
    const DevLut &L = args->lut;
    const int64_t nS = counts[0], nC = counts[1], nP = counts[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool s = bit_at(surv, i), c = bit_at(clone, i), p = bit_at(split, i);
        if (!(s || c || p)) continue;
        const int d = counter[i];
        if (s && !c) {                    // a row kept as stored
            const int64_t o = rank_at(surv, sprefix, i);
            for (int r = 0; r < D; r++) {
                if (r < N_GEO) {
                    Q.geo[r * Q.pitch + o] = P.geo[r * P.pitch + i];
                    Q.m[r * Q.pitch + o] = P.m[r * P.pitch + i];
                    Q.v[r * Q.pitch + o] = P.v[r * P.pitch + i];
                    if (Q.rdir) Q.rdir[r * Q.pitch + o] = P.rdir ? P.rdir[r * P.pitch + i] : 0.f;
                } else {
                    const int64_t a = (r - N_GEO) * P.pitch + i, b = (r - N_GEO) * Q.pitch + o;
                    Q.shw[b] = P.shw[a];
                    Q.shm[b] = P.shm[a];
                    Q.shv[b] = P.shv[a];
                }
            }
            qcounter[o] = (uint8_t)d;
            continue;
        }
        // cloned or split: caught up first
        float cur[N_GEO];
#pragma unroll
        for (int r = 0; r < N_GEO; r++) cur[r] = current<T, OPT>(P, L, r, i, d);
        if (c) {
            // the caught-up row (moments decayed over the d deferred steps) and its zero-moment clone
            const int64_t o = rank_at(surv, sprefix, i), o2 = nS + rank_at(clone, cprefix, i);
            for (int r = 0; r < D; r++) {
                const float w = r < N_GEO ? cur[r] : current<T, OPT>(P, L, r, i, d);
                float m = P.mm(r, i), v = P.vv(r, i);
                if (d) {                   // m b1^d, v b2^d (momentum SGD: b mu^d, v unused)
                    m = L.mom[d - 1] * m;
                    v = L.var[d - 1] * v;
                }
                Q.put(r, o, w, m, v, 0.f);
                const float mq = Q.mm(r, o), vq = Q.vv(r, o);     // the moments as stored: their direction
                if (r < N_GEO && Q.rdir) Q.rdir[r * Q.pitch + o] = restore_dir<OPT>(mq, vq, L.eps);
                Q.put(r, o2, w, 0.f, 0.f, 0.f);
            }
            qcounter[o] = 0;
            qcounter[o2] = 0;
            continue;
        }
        // split: two children, the parent row dropped
        const int64_t k = rank_at(split, pprefix, i);
        float q[4] = {cur[6], cur[7], cur[8], cur[9]};
        const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
        if (qq > 0.f) {
            const float inv = rsqrtf(qq);
            for (int j = 0; j < 4; j++) q[j] *= inv;
        } else {
            q[0] = 1.f;
            q[1] = q[2] = q[3] = 0.f;
        }
        float R[9];
        quat_rot(q, R);
        const float s3[3] = {expf(cur[3]), expf(cur[4]), expf(cur[5])};
        for (int j = 0; j < 2; j++) {
            const int64_t o = nS + nC + j * nP + k;
            float z[3];
            for (int a = 0; a < 3; a++) z[a] = normals[((int64_t)j * 3 + a) * n + i] * s3[a];
            for (int r = 0; r < D; r++) {
                float w = r < N_GEO ? cur[r] : current<T, OPT>(P, L, r, i, d);
                if (r < 3) w = cur[r] + (R[3 * r] * z[0] + R[3 * r + 1] * z[1] + R[3 * r + 2] * z[2]);
                else if (r < 6) w = logf(s3[r - 3] / 1.6f);
                Q.put(r, o, w, 0.f, 0.f, 0.f);
            }
            qcounter[o] = 0;
        }
    }
}

}  // namespace

// Launch the classification and the three compactions; counts[0..2] (device)
// receive the survivor, clone and split counts.
gs_status densify_count(const SceneView &sc, const DevArgs *args, const float *accum, const float *denom,
                        float grad_threshold, float scale_limit, float min_opacity, uint32_t *const masks[3],
                        uint32_t *const prefixes[3], uint32_t *const chunks[3], int *counts, Work &w, cudaStream_t s)
{
    const DensifyRule rule{grad_threshold, scale_limit, min_opacity};
    const int g = w.grid(sc.n, 256, 8);
    with_opt(sc.opt, [&](auto o) {
        constexpr int O = decltype(o)::value;
        if (sc.prec == GS_FP32)
            k_densify_classify<float, O><<<g, 256, 0, s>>>(dplanes<float>(sc), sc.counter, sc.n, args, accum, denom,
                                                           rule, masks[0], masks[1], masks[2]);
        else
            k_densify_classify<__nv_bfloat16, O><<<g, 256, 0, s>>>(dplanes<__nv_bfloat16>(sc), sc.counter, sc.n, args,
                                                                   accum, denom, rule, masks[0], masks[1], masks[2]);
    });
    for (int k = 0; k < 3; k++)
        compact_mask(masks[k], sc.n, chunks[k], false, nullptr, prefixes[k], (int)sc.n, counts + k, w, s);
    return GS_OK;
}

void densify_write(const SceneView &sc, const SceneView &dst, const DevArgs *args, const float *normals,
                   uint32_t *const masks[3], uint32_t *const prefixes[3], const int *counts, Work &w, cudaStream_t s)
{
    const int g = w.grid(sc.n, 256, 8);
    with_opt(sc.opt, [&](auto o) {
        constexpr int O = decltype(o)::value;
        if (sc.prec == GS_FP32)
            k_densify_write<float, O><<<g, 256, 0, s>>>(dplanes<float>(sc), sc.counter, sc.n, sc.D, args, normals,
                                                        masks[0], prefixes[0], masks[1], prefixes[1], masks[2],
                                                        prefixes[2], counts, dplanes<float>(dst), dst.counter);
        else
            k_densify_write<__nv_bfloat16, O><<<g, 256, 0, s>>>(
                dplanes<__nv_bfloat16>(sc), sc.counter, sc.n, sc.D, args, normals, masks[0], prefixes[0], masks[1],
                prefixes[1], masks[2], prefixes[2], counts, dplanes<__nv_bfloat16>(dst), dst.counter);
    });
}

}  // namespace gs
