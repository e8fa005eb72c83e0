// gs_cpu_opt.cu -- host-core optimizer of the offloaded configuration
// (§4.2.2 parameter forwarding, §4.3 deferred update), OpenMP over members.
// Same update as the device kernels (Eq. 1 with the restore tables of
// Fig. 10 / reading of the deferred catch-up, AdamW decay, momentum SGD), in
// FP32 with IEEE square root and division.
#include <omp.h>

#include <algorithm>
#include <cmath>

#include "cpu_opt.hpp"

namespace gs {
namespace {

constexpr int64_t CHUNK = 4096;   // members per work item: each thread walks the planes of its chunk

template <int OPT> inline float h_dir(float m, float v, float eps)
{
    return OPT == GS_OPT_SGDM ? m : m / (std::sqrt(v) + eps);
}

// The value of a parameter whose last d updates were deferred (Eq. 3 with the
// tables of step L.step); AdamW also decays over the deferred steps.
template <int OPT> inline float h_restore(float w, float m, float v, int d, int grp, const DevLut &L)
{
    if (!d) return w;
    const float dir = h_dir<OPT>(m, v, L.eps);
    if (OPT == GS_OPT_ADAMW) return std::fma(-L.param[grp][d], dir, L.decay[grp][d] * w);
    return std::fma(-L.param[grp][d], dir, w);
}

// Catch-up over d deferred steps, then one step with gradient g (Eq. 1).
template <int OPT> inline void h_step(float &w, float &m, float &v, float g, int d, int grp, const DevLut &L)
{
    const float m_new = L.mom[d] * m + L.omb1 * g;
    if (OPT == GS_OPT_SGDM) {
        w = h_restore<OPT>(w, m, v, d, grp, L) - L.step_size[grp] * m_new;
        m = m_new;
        return;
    }
    const float v_new = L.var[d] * v + L.omb2 * g * g;
    const float wr = h_restore<OPT>(w, m, v, d, grp, L);
    const float denom = std::sqrt(v_new) * L.inv_bias_corr + L.eps;
    const float ws = OPT == GS_OPT_ADAMW ? L.wdf[grp] * wr : wr;
    w = ws - L.step_size[grp] * (m_new / denom);
    m = m_new;
    v = v_new;
}

// Gradient row of each member of uids[u0..u1): position in vids, or -1.
inline void grad_rows(const int32_t *uids, int64_t u0, int64_t u1, const int32_t *vids, int64_t n_vis, int64_t *row)
{
    int64_t k = std::lower_bound(vids, vids + n_vis, uids[u0]) - vids;
    for (int64_t u = u0; u < u1; u++) {
        const int32_t i = uids[u];
        while (k < n_vis && vids[k] < i) k++;
        row[u - u0] = (k < n_vis && vids[k] == i) ? k : -1;
    }
}

template <int OPT> void deferred_step(const HostPlanes &P, const CpuUpdate &U, int threads)
{
    const int64_t nch = (U.n_upd + CHUNK - 1) / CHUNK;
#pragma omp parallel num_threads(threads)
    {
        int64_t row[CHUNK];
#pragma omp for schedule(dynamic, 4)
        for (int64_t c = 0; c < nch; c++) {
            const int64_t u0 = c * CHUNK, u1 = std::min(U.n_upd, u0 + CHUNK);
            grad_rows(U.uids, u0, u1, U.vids, U.n_vis, row);
            for (int r = 0; r < P.planes; r++) {
                const int grp = lr_group(P.plane0 + r);
                float *w = P.w + r * P.pitch, *m = P.m + r * P.pitch, *v = P.v + r * P.pitch;
                const float *g = U.grad + r * U.gpitch;
                for (int64_t u = u0; u < u1; u++) {
                    const int64_t i = U.uids[u], k = row[u - u0];
                    h_step<OPT>(w[i], m[i], v[i], k >= 0 ? g[k] : 0.f, U.udelay[u], grp, U.lut);
                }
            }
        }
    }
}

template <int OPT>
void forward(const HostPlanes &P, const int32_t *ids, const uint8_t *cnt, int64_t n, const CpuUpdate *U,
             const DevLut &Ln, float *out, int64_t opitch, int threads)
{
    const int64_t nch = (n + CHUNK - 1) / CHUNK;
#pragma omp parallel num_threads(threads)
    {
        int64_t urow[CHUNK], grow[CHUNK];
#pragma omp for schedule(dynamic, 4)
        for (int64_t c = 0; c < nch; c++) {
            const int64_t k0 = c * CHUNK, k1 = std::min(n, k0 + CHUNK);
            // pending members among ids[k0..k1) (counter 0): their place in
            // the update set and their gradient row
            int64_t u = U && U->n_upd ? std::lower_bound(U->uids, U->uids + U->n_upd, ids[k0]) - U->uids : 0;
            int64_t q = U && U->n_vis ? std::lower_bound(U->vids, U->vids + U->n_vis, ids[k0]) - U->vids : 0;
            for (int64_t k = k0; k < k1; k++) {
                urow[k - k0] = grow[k - k0] = -1;
                if (!U || cnt[k]) continue;
                const int32_t i = ids[k];
                while (u < U->n_upd && U->uids[u] < i) u++;
                while (q < U->n_vis && U->vids[q] < i) q++;
                if (u < U->n_upd && U->uids[u] == i) urow[k - k0] = u;
                if (q < U->n_vis && U->vids[q] == i) grow[k - k0] = q;
            }
            for (int r = 0; r < P.planes; r++) {
                const int grp = lr_group(P.plane0 + r);
                const float *w = P.w + r * P.pitch, *m = P.m + r * P.pitch, *v = P.v + r * P.pitch;
                float *o = out + r * opitch;
                for (int64_t k = k0; k < k1; k++) {
                    const int64_t i = ids[k];
                    float wi = w[i], mi = m[i], vi = v[i];
                    if (cnt[k]) {
                        wi = h_restore<OPT>(wi, mi, vi, cnt[k], grp, Ln);
                    } else if (urow[k - k0] >= 0) {
                        const int64_t gq = grow[k - k0];
                        h_step<OPT>(wi, mi, vi, gq >= 0 ? U->grad[r * U->gpitch + gq] : 0.f, U->udelay[urow[k - k0]],
                                    grp, U->lut);
                    }
                    o[k] = wi;
                }
            }
        }
    }
}

}  // namespace

void cpu_deferred_step(const HostPlanes &P, const CpuUpdate &U, int threads)
{
    if (U.n_upd <= 0) return;
    if (threads <= 0) threads = omp_get_max_threads();
    switch (U.opt) {
    case GS_OPT_ADAMW: deferred_step<GS_OPT_ADAMW>(P, U, threads); break;
    case GS_OPT_SGDM: deferred_step<GS_OPT_SGDM>(P, U, threads); break;
    default: deferred_step<GS_OPT_ADAM>(P, U, threads); break;
    }
}

void cpu_forward(const HostPlanes &P, const int32_t *ids, const uint8_t *cnt, int64_t n, const CpuUpdate *U,
                 const DevLut &Ln, int opt, float *out, int64_t opitch, int threads)
{
    if (n <= 0) return;
    if (threads <= 0) threads = omp_get_max_threads();
    switch (opt) {
    case GS_OPT_ADAMW: forward<GS_OPT_ADAMW>(P, ids, cnt, n, U, Ln, out, opitch, threads); break;
    case GS_OPT_SGDM: forward<GS_OPT_SGDM>(P, ids, cnt, n, U, Ln, out, opitch, threads); break;
    default: forward<GS_OPT_ADAM>(P, ids, cnt, n, U, Ln, out, opitch, threads); break;
    }
}

}  // namespace gs
