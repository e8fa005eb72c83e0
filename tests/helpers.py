"""Shared helpers of the GPU parity tests: inputs rounded to what the GPU sees,
oracle runs on those inputs, and comparison rules for discrete decisions."""
from __future__ import annotations

import copy

import numpy as np

# A discrete decision (cull, rect edge, alpha threshold, square test, T stop)
# whose FP64 margin is below this relative distance may legitimately go the
# other way in FP32; such Gaussians / pixels are excluded and counted.
TIE_TOL = 1e-5


def cam_f32(cam):
    """The camera with every field rounded to float32, as the GPU receives it."""
    c = copy.copy(cam)
    c.R = np.asarray(cam.R, np.float32).astype(np.float64)
    c.t = np.asarray(cam.t, np.float32).astype(np.float64)
    for k in ("fx", "fy", "cx", "cy", "near", "far"):
        setattr(c, k, float(np.float32(getattr(cam, k))))
    return c


def hp32(orc, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-15, max_defer=15):
    """Oracle Adam hyper-parameters rounded to float32, as the C ABI carries them."""
    lr32 = np.asarray(np.broadcast_to(lr, (6,)), np.float32).astype(np.float64)
    r = lambda x: float(np.float32(x))
    return orc.AdamHyper(lr=lr32, beta1=r(beta1), beta2=r(beta2), eps=r(eps), max_defer=max_defer)


def f32(params):
    return np.asarray(params, np.float32).astype(np.float64)


def rel_group_error(g_gpu, g_ref, rows):
    """||gpu - ref|| / ||ref|| over a group of parameter rows."""
    a = g_gpu[rows].ravel()
    b = g_ref[rows].ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


GROUPS = {"mean": slice(0, 3), "log_scale": slice(3, 6), "quat": slice(6, 10), "opacity": slice(10, 11),
          "sh_dc": slice(11, 14), "sh_rest": slice(14, None)}


def check_lists(gpu_tiles, gpu_gids, oracle_tiles, oracle_gids, depth_bits, exclude):
    """GPU (tile, Gaussian id) sequence against the oracle's.  Keys of excluded
    Gaussians are dropped from both; within a tile, neighbours may differ in
    order only when their float32 depths are within 2 ulp."""
    keep_g = ~np.isin(gpu_gids, exclude)
    keep_o = ~np.isin(oracle_gids, exclude)
    gt, gg = gpu_tiles[keep_g], gpu_gids[keep_g]
    ot, og = oracle_tiles[keep_o], oracle_gids[keep_o]
    assert gt.shape == ot.shape, (gt.shape, ot.shape)
    np.testing.assert_array_equal(gt, ot)
    if np.array_equal(gg, og):
        return 0
    bad = np.nonzero(gg != og)[0]
    # allowed only as swaps of near-equal depths inside one tile
    for p in bad:
        t = gt[p]
        lo = p
        while lo > 0 and gt[lo - 1] == t:
            lo -= 1
        hi = p
        while hi + 1 < len(gt) and gt[hi + 1] == t:
            hi += 1
        assert sorted(gg[lo:hi + 1]) == sorted(og[lo:hi + 1])
        d = depth_bits[gg[p]].astype(np.int64)
        e = depth_bits[og[p]].astype(np.int64)
        assert abs(d - e) <= 2, (p, gg[p], og[p], d, e)
    return len(bad)


def pixel_exclusions(r, gpu_ids=None):
    """Pixels whose value may legitimately differ between FP32 and FP64: a
    near-tie among the decisions that can change the pixel (square test of a
    contributing Gaussian, the 1/255 floor, the transmittance stop), the ring
    of pixels where a Gaussian's 3-sigma square test flips when its integer
    radius is a near-tie, or the whole square of a Gaussian whose keep decision
    differs (a near-tie of the cull)."""
    ex = r["margin"] < TIE_TOL
    sp = r["splats"]
    H, W = ex.shape
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    ring = (sp["radius_margin"] < TIE_TOL) & (sp["keep"] == 1)
    whole = np.zeros_like(ring)
    if gpu_ids is not None:
        whole[np.setxor1d(gpu_ids, np.nonzero(sp["keep"])[0])] = True
    for i in np.nonzero(ring | whole)[0]:
        mx, my = sp["mean2d"][i]
        rr = sp["radius"][i]
        if not (np.isfinite(mx) and np.isfinite(my) and rr > 0):
            continue
        dist = np.maximum(np.abs(xs - mx), np.abs(ys - my))
        if whole[i]:
            ex |= dist <= rr + 1.5
        else:
            ex |= np.abs(dist - rr) <= 1.01
    return ex


def cancellation_bound(sp, H, W, u=2.0 ** -24):
    """Per-pixel bound on the FP32 compositing error that the cancellation in
    sigma = 1/2 (A dx^2 + C dy^2) + B dx dy allows: every kept splat whose
    3-sigma square covers the pixel adds 8 u sigma_abs, sigma_abs = (|A| +
    2|B| + |C|) r^2 / 2 (long thin splats have large ones)."""
    keep = np.nonzero(sp["keep"] == 1)[0]
    con, rad = sp["conic"][keep], sp["radius"][keep]
    sabs = 0.5 * (np.abs(con[:, 0]) + 2 * np.abs(con[:, 1]) + np.abs(con[:, 2])) * rad ** 2
    out = np.zeros((H, W))
    for j in np.nonzero(8 * u * sabs > 1e-7)[0]:
        mx, my = sp["mean2d"][keep[j]]
        r = rad[j]
        x0, x1 = max(0, int(np.floor(mx - r - 0.5))), min(W, int(np.ceil(mx + r + 0.5)))
        y0, y1 = max(0, int(np.floor(my - r - 0.5))), min(H, int(np.ceil(my + r + 0.5)))
        if x0 < x1 and y0 < y1:
            out[y0:y1, x0:x1] += 8 * u * sabs[j]
    return out
