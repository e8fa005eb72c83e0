// gs_cpu_opt.cu -- host-core optimizer of the offloaded configuration
// (§4.2.2 parameter forwarding, §4.3 deferred update), OpenMP over members.
// Same update as the device kernels (Eq. 1, the deferred catch-up with the
// restore tables of Fig. 10, the AdamW decay, momentum SGD), in FP32 with IEEE
// square root and division.  The host arrays are Gaussian-major (one row of
// SH values per Gaussian), so a member's update reads and writes a few
// contiguous cache lines per array, as a per-Gaussian tensor layout on the
// host would.
#include <omp.h>

#include <algorithm>
#include <cmath>

#include "cpu_opt.hpp"

namespace gs {
namespace {

constexpr int64_t CHUNK = 512;      // rows per work item (a chunk's rows of w, m, v stay in the core's cache)
constexpr int MAXP = 64;            // longest row handled (48 SH values at degree 3)

template <int OPT> inline float h_dir(float m, float v, float eps)
{
    return OPT == GS_OPT_SGDM ? m : m / (std::sqrt(v) + eps);
}

// The value of a parameter whose last d updates were deferred (Eq. 3 with the
// tables of step L.step); AdamW also decays over the deferred steps.  Plain
// multiply and add: the host build targets the baseline x86-64 ISA, where
// std::fma is a library call.
template <int OPT> inline float h_restore(float w, float m, float v, int d, float plut, float dec, float eps)
{
    if (!d) return w;
    const float dir = h_dir<OPT>(m, v, eps);
    if (OPT == GS_OPT_ADAMW) return dec * w - plut * dir;
    return w - plut * dir;
}

// Catch-up over d deferred steps, then one step with gradient g (Eq. 1).
template <int OPT> inline void h_step(float &w, float &m, float &v, float g, int d, int grp, const DevLut &L)
{
    const float m_new = L.mom[d] * m + L.omb1 * g;
    const float wr = h_restore<OPT>(w, m, v, d, L.param[grp][d], L.decay[grp][d], L.eps);
    if (OPT == GS_OPT_SGDM) {
        w = wr - L.step_size[grp] * m_new;
        m = m_new;
        return;
    }
    const float v_new = L.var[d] * v + L.omb2 * g * g;
    const float denom = std::sqrt(v_new) * L.inv_bias_corr + L.eps;
    const float ws = OPT == GS_OPT_ADAMW ? L.wdf[grp] * wr : wr;
    w = ws - L.step_size[grp] * (m_new / denom);
    m = m_new;
    v = v_new;
}

// Runs of consecutive rows in one learning-rate group: [b[j], b[j + 1]) has group grp[j].
struct GroupRuns {
    int n = 0;
    int b[8], grp[8];
};

// Catch-up and step of values [r0, r1) of one Gaussian's row, all in one
// group (delay and tables fixed over the run: a loop the compiler vectorises).
template <int OPT>
inline void step_span(float *w, float *m, float *v, const float *g, int r0, int r1, int d, int grp, const DevLut &L)
{
#pragma omp simd
    for (int r = r0; r < r1; r++) h_step<OPT>(w[r], m[r], v[r], g ? g[r] : 0.f, d, grp, L);
}

template <int OPT>
inline void step_row(float *w, float *m, float *v, const float *g, int d, const GroupRuns &R, const DevLut &L)
{
    for (int j = 0; j < R.n; j++) step_span<OPT>(w, m, v, g, R.b[j], R.b[j + 1], d, R.grp[j], L);
}

// Position in vids (ascending) of each of ids[0..n) (ascending), or -1.
inline void match_rows(const int32_t *ids, int64_t n, const int32_t *vids, int64_t n_vis, int64_t *row)
{
    if (n <= 0) return;
    int64_t k = std::lower_bound(vids, vids + n_vis, ids[0]) - vids;
    for (int64_t j = 0; j < n; j++) {
        while (k < n_vis && vids[k] < ids[j]) k++;
        row[j] = (k < n_vis && vids[k] == ids[j]) ? k : -1;
    }
}

inline GroupRuns runs_of(const HostPlanes &P)
{
    GroupRuns R;
    for (int r = 0; r < P.planes; r++) {
        const int g = lr_group(P.plane0 + r);
        if (R.n == 0 || R.grp[R.n - 1] != g) {
            R.b[R.n] = r;
            R.grp[R.n++] = g;
        }
    }
    R.b[R.n] = P.planes;
    return R;
}

template <int OPT> void deferred_step(const HostPlanes &P, const CpuUpdate &U, int threads)
{
    const int64_t nch = (U.n_upd + CHUNK - 1) / CHUNK;
    const GroupRuns R = runs_of(P);
#pragma omp parallel num_threads(threads)
    {
        int64_t row[CHUNK];
#pragma omp for schedule(dynamic, 8)
        for (int64_t c = 0; c < nch; c++) {
            const int64_t u0 = c * CHUNK, u1 = std::min(U.n_upd, u0 + CHUNK);
            match_rows(U.uids + u0, u1 - u0, U.vids, U.n_vis, row);
            for (int64_t u = u0; u < u1; u++) {
                const int64_t o = (int64_t)U.uids[u] * P.row, k = row[u - u0];
                step_row<OPT>(P.w + o, P.m + o, P.v + o, k >= 0 ? U.grad + k * U.grow : nullptr, U.udelay[u], R,
                              U.lut);
            }
        }
    }
}

template <int OPT>
void forward(const HostPlanes &P, const int32_t *ids, const uint8_t *cnt, int64_t n, const CpuUpdate *U,
             const DevLut &Ln, float *out, int64_t opitch, int threads)
{
    const int64_t nch = (n + CHUNK - 1) / CHUNK;
    const GroupRuns R = runs_of(P);
#pragma omp parallel num_threads(threads)
    {
        int64_t urow[CHUNK], grow[CHUNK];
        float wt[MAXP], mt[MAXP], vt[MAXP];
#pragma omp for schedule(dynamic, 8)
        for (int64_t c = 0; c < nch; c++) {
            const int64_t k0 = c * CHUNK, k1 = std::min(n, k0 + CHUNK);
            // pending members among ids[k0..k1): their place in the update set
            // and their gradient row
            if (U) {
                match_rows(ids + k0, k1 - k0, U->uids, U->n_upd, urow);
                match_rows(ids + k0, k1 - k0, U->vids, U->n_vis, grow);
            }
            for (int64_t k = k0; k < k1; k++) {
                const int64_t o = (int64_t)ids[k] * P.row;
                const float *w = P.w + o, *m = P.m + o, *v = P.v + o;
                const int d = cnt[k];
                if (d) {
                    for (int j = 0; j < R.n; j++) {
                        const float plut = Ln.param[R.grp[j]][d], dec = Ln.decay[R.grp[j]][d];
#pragma omp simd
                        for (int r = R.b[j]; r < R.b[j + 1]; r++) wt[r] = h_restore<OPT>(w[r], m[r], v[r], d, plut, dec, Ln.eps);
                    }
                    for (int r = 0; r < P.planes; r++) out[r * opitch + k] = wt[r];
                } else if (U && urow[k - k0] >= 0) {
                    for (int r = 0; r < P.planes; r++) {
                        wt[r] = w[r];
                        mt[r] = m[r];
                        vt[r] = v[r];
                    }
                    const int64_t q = grow[k - k0];
                    step_row<OPT>(wt, mt, vt, q >= 0 ? U->grad + q * U->grow : nullptr, U->udelay[urow[k - k0]], R,
                                  U->lut);
                    for (int r = 0; r < P.planes; r++) out[r * opitch + k] = wt[r];
                } else {
                    for (int r = 0; r < P.planes; r++) out[r * opitch + k] = w[r];
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
