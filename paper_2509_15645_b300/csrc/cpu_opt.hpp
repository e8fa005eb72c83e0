// cpu_opt.hpp -- the optimizer of the paper's offloaded configuration on the
// host cores (§4.2.2 parameter forwarding, §4.3 deferred update, OpenMP).
// Planes of a parameter range live in host memory; the update-set members of
// a step, their delays and the gradients of the Gaussians that had one come
// from the device.  Host code only (no kernels).
#pragma once
#include <cstdint>

#include "gs_internal.cuh"

namespace gs {

// Rows [plane0, plane0 + planes) of the parameter vector, Gaussian-major:
// the value of row plane0 + r of Gaussian i at i * row + r of each array.
struct HostPlanes {
    float *w, *m, *v;
    int64_t row;            // floats per Gaussian, >= planes
    int plane0, planes;     // planes <= 64
};

// One step's update, held until the host applies it: members (ascending ids)
// with their delays, the Gaussians with a gradient row (ascending ids) and
// those rows (row k, for vids[k], at grad + k * grow), the step's tables.
struct CpuUpdate {
    const int32_t *uids = nullptr;
    const uint8_t *udelay = nullptr;
    int64_t n_upd = 0;
    const int32_t *vids = nullptr;
    const float *grad = nullptr;
    int64_t n_vis = 0, grow = 0;
    DevLut lut{};
    int opt = GS_OPT_ADAM;
};

// Apply `U` to the planes (the lazy update of §4.2.2 step 5): each member is
// caught up over its delay and stepped with its gradient (zero without a row).
void cpu_deferred_step(const HostPlanes &P, const CpuUpdate &U, int threads);

// Parameter forwarding (§4.2.2 step 1): the current values of Gaussians
// ids[0..n) (ascending) for the next step, written plane-major to
// out[r * opitch + k] (the layout the device reads), without
// changing the planes.  cnt[k] is Gaussian ids[k]'s defer counter at the next
// step: > 0 restores over that many deferred steps with the next step's tables
// `Ln`; 0 applies the member's pending update `U` (if it is in U's update set,
// else the stored value is current).  U may be null (nothing pending).
void cpu_forward(const HostPlanes &P, const int32_t *ids, const uint8_t *cnt, int64_t n, const CpuUpdate *U,
                 const DevLut &Ln, int opt, float *out, int64_t opitch, int threads);

}  // namespace gs
