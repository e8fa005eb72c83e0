"""ctypes front end of the FP64 C oracle (``gs_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  Arrays are
numpy float64; parameters use the [D][n] structure-of-arrays layout of
``synth.scenes``.  Functions follow GS-Scale §2.4 (render steps 1-5), Eq. 1
(eager Adam), Eqs. 2-3 with the pseudocode of Fig. 10 (deferred Adam) and §4.4
(balance-aware image splitting).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

c_i64, c_i32, c_dbl = C.c_int64, C.c_int32, C.c_double
P_DBL = C.POINTER(C.c_double)


class OrcCamera(C.Structure):
    _fields_ = [("R", c_dbl * 9), ("t", c_dbl * 3), ("fx", c_dbl), ("fy", c_dbl), ("cx", c_dbl),
                ("cy", c_dbl), ("near_z", c_dbl), ("far_z", c_dbl), ("width", c_i32),
                ("height", c_i32), ("tile_w", c_i32), ("tile_h", c_i32)]


SPLAT = np.dtype([("keep", "<i4"), ("rect", "<i4", 4), ("clampx", "<i4"), ("clampy", "<i4"),
                  ("rgb_clamped", "<i4", 3), ("pad", "<i4"), ("depth", "<f8"), ("mean2d", "<f8", 2),
                  ("cov2d", "<f8", 3), ("conic", "<f8", 3), ("radius", "<f8"), ("opacity", "<f8"),
                  ("rgb", "<f8", 3), ("margin", "<f8"), ("depth_f32", "<f8"),
                  ("radius_margin", "<f8")], align=True)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _lib.orc_count_keys.restype = c_i64
        _lib.orc_loss_l1.restype = c_dbl
        _lib.orc_splat_size.restype = C.c_int
        _lib.orc_num_threads.restype = C.c_int
        assert _lib.orc_splat_size() == SPLAT.itemsize, "splat layout mismatch"
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def n_params(deg: int) -> int:
    return 11 + 3 * (deg + 1) ** 2


def camera(cam, tile=(16, 16)) -> OrcCamera:
    """Convert a ``synth.scenes.Camera`` (float64 fields) to the oracle's struct."""
    c = OrcCamera()
    R = np.asarray(cam.R, np.float64).reshape(9)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(cam.t[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_z, c.far_z = float(cam.near), float(cam.far)
    c.width, c.height = int(cam.width), int(cam.height)
    c.tile_w, c.tile_h = int(tile[0]), int(tile[1])
    return c


def tiles_of(oc: OrcCamera):
    return (oc.width + oc.tile_w - 1) // oc.tile_w, (oc.height + oc.tile_h - 1) // oc.tile_h


def _f64(params) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(params, dtype=np.float64))


def project(params, deg: int, oc: OrcCamera) -> np.ndarray:
    """Step 1 of §2.4 for every Gaussian: returns the SPLAT record array."""
    P = _f64(params)
    n = P.shape[1]
    out = np.zeros(n, SPLAT)
    lib().orc_project(c_i64(n), C.c_int(deg), _p(P), c_i64(n), C.byref(oc), _p(out))
    return out


def build_lists(splats: np.ndarray, oc: OrcCamera):
    """Step 2 of §2.4: sorted (tile, Gaussian id) keys and per-tile ranges.  A
    pair is kept when the Gaussian reaches alpha >= 1/255 in the tile
    (``tile_reach``)."""
    n = splats.shape[0]
    K = lib().orc_count_keys(c_i64(n), _p(splats), C.byref(oc))
    tx, ty = tiles_of(oc)
    key_tile = np.zeros(max(K, 1), np.int32)
    key_gid = np.zeros(max(K, 1), np.int64)
    ranges = np.zeros(2 * tx * ty, np.int64)
    lib().orc_build_lists(c_i64(n), _p(splats), C.byref(oc), _p(key_tile), _p(key_gid), _p(ranges))
    return key_tile[:K], key_gid[:K], ranges.reshape(-1, 2)


def tile_reach(splats, oc: OrcCamera, gids, tiles, ext=0.0):
    """Largest o exp(-sigma) of Gaussian gids[k] over the box of tile tiles[k]'s
    pixel centres inside its 3-sigma square widened by ``ext`` pixels (0 where
    they do not meet): the quantity the list filter compares with 1/255."""
    g = np.ascontiguousarray(gids, np.int64).ravel()
    t = np.ascontiguousarray(tiles, np.int64).ravel()
    assert g.shape == t.shape
    out = np.zeros(g.shape[0])
    lib().orc_tile_reach_many(c_i64(g.shape[0]), _p(splats), C.byref(oc), _p(g), _p(t), c_dbl(ext), _p(out))
    return out


def composite(splats, oc: OrcCamera, key_gid, ranges, bg=(0.0, 0.0, 0.0)):
    """Step 3 of §2.4.  Returns image [3][H][W], contributor counts, final T,
    the per-pixel decision margin and a hash of each pixel's contributor
    sequence (ids and alpha-clamp states)."""
    H, W = oc.height, oc.width
    img = np.zeros((3, H, W))
    ncon = np.zeros((H, W), np.int32)
    Tf = np.zeros((H, W))
    mg = np.zeros((H, W))
    hs = np.zeros((H, W), np.uint64)
    bgv = np.asarray(bg, np.float64)
    kg = np.ascontiguousarray(key_gid, np.int64)
    rg = np.ascontiguousarray(ranges, np.int64)
    lib().orc_composite(c_i64(splats.shape[0]), _p(splats), C.byref(oc), _p(kg), _p(rg), _p(bgv),
                        _p(img), _p(ncon), _p(Tf), _p(mg), _p(hs))
    return img, ncon, Tf, mg, hs


def composite_brute(splats, oc: OrcCamera, bg=(0.0, 0.0, 0.0)):
    img = np.zeros((3, oc.height, oc.width))
    bgv = np.asarray(bg, np.float64)
    lib().orc_composite_brute(c_i64(splats.shape[0]), _p(splats), C.byref(oc), _p(bgv), _p(img))
    return img


def loss_l1(image, target):
    """Step 4 of §2.4 with L1: (loss, dL/dimage)."""
    img = np.ascontiguousarray(image, np.float64)
    tgt = np.ascontiguousarray(target, np.float64)
    d = np.zeros_like(img)
    loss = lib().orc_loss_l1(c_i64(img.size), _p(img), _p(tgt), _p(d))
    return loss, d


def backward(params, deg, oc, splats, key_gid, ranges, dimage, bg=(0.0, 0.0, 0.0)):
    """Step 5 of §2.4: dL/dparams [D][n] and the per-Gaussian screen-space
    sums [n][9] = (mean2d x, y, conic A, B, C, opacity, r, g, b)."""
    P = _f64(params)
    D, n = P.shape
    grad = np.zeros((D, n))
    sg = np.zeros((n, 9))
    bgv = np.asarray(bg, np.float64)
    di = np.ascontiguousarray(dimage, np.float64)
    lib().orc_backward(c_i64(n), C.c_int(deg), _p(P), c_i64(n), C.byref(oc), _p(splats),
                       _p(np.ascontiguousarray(key_gid, np.int64)),
                       _p(np.ascontiguousarray(ranges, np.int64)), _p(bgv), _p(di), _p(grad), _p(sg))
    return grad, sg


def render(params, deg, cam, tile=(16, 16), bg=(0.0, 0.0, 0.0)):
    """Project, build lists and composite one view."""
    oc = camera(cam, tile)
    sp = project(params, deg, oc)
    kt, kg, rg = build_lists(sp, oc)
    img, ncon, Tf, mg, hs = composite(sp, oc, kg, rg, bg)
    return dict(cam=oc, splats=sp, key_tile=kt, key_gid=kg, ranges=rg, image=img, n_contrib=ncon,
                T_final=Tf, margin=mg, decision_hash=hs)


def render_loss_backward(params, deg, cam, target, tile=(16, 16)):
    """One forward + L1 loss + backward; returns the render dict plus loss and grads."""
    r = render(params, deg, cam, tile)
    loss, dimg = loss_l1(r["image"], target)
    grad, sg = backward(params, deg, r["cam"], r["splats"], r["key_gid"], r["ranges"], dimg)
    r.update(loss=loss, dimage=dimg, grad=grad, splat_grad=sg)
    return r


def sh_basis(deg, direction):
    Y = np.zeros(16)
    dY = np.zeros(48)
    d = np.ascontiguousarray(direction, np.float64)
    lib().orc_sh_basis(C.c_int(deg), _p(d), _p(Y), _p(dY))
    return Y, dY.reshape(16, 3)


# ---------------------------------------------------------------- Adam

class AdamHyper:
    def __init__(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-15, max_defer=15):
        self.lr = np.full(6, lr, np.float64) if np.isscalar(lr) else np.asarray(lr, np.float64)
        self.beta1, self.beta2, self.eps, self.max_defer = beta1, beta2, eps, max_defer


def adam_eager(w, m, v, g, t, hp: AdamHyper):
    """Eq. 1 at step t on every value (in place)."""
    D, n = w.shape
    lib().orc_adam_eager(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(m), _p(v),
                         _p(np.ascontiguousarray(g, np.float64)), C.c_int(t), _p(hp.lr),
                         c_dbl(hp.beta1), c_dbl(hp.beta2), c_dbl(hp.eps))


def adam_lut(t, lr, hp: AdamHyper):
    K = hp.max_defer + 1
    pl, ml, vl = np.zeros(K), np.zeros(K), np.zeros(K)
    lib().orc_adam_lut(C.c_int(t), c_dbl(lr), c_dbl(hp.beta1), c_dbl(hp.beta2), C.c_int(hp.max_defer),
                       _p(pl), _p(ml), _p(vl))
    return pl, ml, vl


def adam_deferred(w, m, v, counter, ids, g_compact, t, hp: AdamHyper, mode=0, geo_eager=False):
    """Deferred update at step t (in place).  mode 0: lookup tables (Eq. 3),
    mode 1: exact replay of the zero-gradient steps."""
    D, n = w.shape
    ids = np.ascontiguousarray(ids, np.int32)
    gc = np.ascontiguousarray(g_compact, np.float64).reshape(D, ids.shape[0])
    assert counter.dtype == np.uint8
    lib().orc_adam_deferred(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(m), _p(v), _p(counter), _p(ids),
                            c_i64(ids.shape[0]), _p(gc), C.c_int(t), _p(hp.lr), c_dbl(hp.beta1),
                            c_dbl(hp.beta2), c_dbl(hp.eps), C.c_int(hp.max_defer), C.c_int(mode),
                            C.c_int(int(geo_eager)))


def adam_materialize(w, m, v, counter, t_done, hp: AdamHyper, mode=0, geo_eager=False):
    D, n = w.shape
    wo, mo, vo = np.zeros_like(w), np.zeros_like(m), np.zeros_like(v)
    lib().orc_adam_materialize(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(m), _p(v), _p(counter),
                               C.c_int(t_done), _p(hp.lr), c_dbl(hp.beta1), c_dbl(hp.beta2),
                               c_dbl(hp.eps), C.c_int(hp.max_defer), C.c_int(mode),
                               C.c_int(int(geo_eager)), _p(wo), _p(mo), _p(vo))
    return wo, mo, vo


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """OpenMP threads of the following oracle calls (timing only)."""
    lib().orc_set_num_threads(C.c_int(int(n)))


def depth_bits(depth_f64) -> np.ndarray:
    return np.asarray(depth_f64, np.float64).astype(np.float32).view(np.uint32)




# ---------------------------------------------------------------------------- image splitting (§4.4)

def split_counts(splats, axis: int, at: int):
    """Visible-Gaussian counts of the two regions of a view split at tile
    boundary ``at`` along ``axis`` (0: tile columns [0, at) and [at, tiles_x);
    1: tile rows).  Each region culls on its own (§4.4): a Gaussian counts for
    a region when it survives the view's cull and its tile rectangle (from
    ``project``) reaches the region's tiles, so one that straddles the
    boundary counts for both."""
    keep = splats["keep"] == 1
    first, last = splats["rect"][:, 2 * axis], splats["rect"][:, 2 * axis + 1]    # half-open tile range
    return int(np.count_nonzero(keep & (first < at))), int(np.count_nonzero(keep & (last > at)))


def balance_split(splats, oc: OrcCamera, axis: int, steps: int = 5):
    """Balance-aware split point of §4.4 (the paper: 5 steps, once before
    training).  Start at the middle tile boundary, cull both sides, and move
    the boundary into the side with more visible Gaussians by halving the
    remaining interval each step; boundaries stay inside (0, tiles).  Returns
    (boundary in tiles, counts of both regions there)."""
    tiles = tiles_of(oc)[axis]
    assert tiles >= 2, "a split needs two tiles along the axis"

    def inside(x):
        return min(max(x, 1), tiles - 1)

    lo, hi = 0, tiles
    for _ in range(steps):
        at = inside((lo + hi) // 2)
        first, second = split_counts(splats, axis, at)
        if first > second:
            hi = at          # the first region is fuller: shrink it
        else:
            lo = at
    at = inside((lo + hi) // 2)
    return at, split_counts(splats, axis, at)


# ---------------------------------------------------------------------------- AdamW, SGD with momentum (§4.3)

def adamw_lut(t, lr, hp: AdamHyper, wd):
    """AdamW restore tables at step t: (wlut [MAX+1], decay [MAX+1])."""
    K = hp.max_defer + 1
    wl, dec = np.zeros(K), np.zeros(K)
    lib().orc_adamw_lut(C.c_int(t), c_dbl(lr), c_dbl(hp.beta1), c_dbl(hp.beta2), c_dbl(wd), C.c_int(hp.max_defer),
                        _p(wl), _p(dec))
    return wl, dec


def sgdm_lut(lr, mu, max_defer=15):
    """Momentum-SGD restore tables: (slut [MAX+1], mom [MAX+1] = mu^(d+1))."""
    sl, mo = np.zeros(max_defer + 1), np.zeros(max_defer + 1)
    lib().orc_sgdm_lut(c_dbl(lr), c_dbl(mu), C.c_int(max_defer), _p(sl), _p(mo))
    return sl, mo


def adamw_eager(w, m, v, g, t, hp: AdamHyper, wd):
    """One AdamW step (decoupled weight decay wd) on every value (in place)."""
    D, n = w.shape
    lib().orc_adamw_eager(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(m), _p(v),
                          _p(np.ascontiguousarray(g, np.float64)), C.c_int(t), _p(hp.lr), c_dbl(hp.beta1),
                          c_dbl(hp.beta2), c_dbl(hp.eps), c_dbl(wd))


def sgdm_eager(w, b, g, lr, mu):
    """One step of SGD with momentum mu (buffer b, no dampening) on every value (in place)."""
    D, n = w.shape
    lr = np.full(6, lr, np.float64) if np.isscalar(lr) else np.asarray(lr, np.float64)
    lib().orc_sgdm_eager(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(b), _p(np.ascontiguousarray(g, np.float64)),
                         _p(lr), c_dbl(mu))


def adamw_deferred(w, m, v, counter, ids, g_compact, t, hp: AdamHyper, wd, mode=0):
    """Deferred AdamW at step t (in place); mode 0 tables, mode 1 replay."""
    D, n = w.shape
    ids = np.ascontiguousarray(ids, np.int32)
    gc = np.ascontiguousarray(g_compact, np.float64).reshape(D, ids.shape[0])
    assert counter.dtype == np.uint8
    lib().orc_adamw_deferred(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(m), _p(v), _p(counter), _p(ids),
                             c_i64(ids.shape[0]), _p(gc), C.c_int(t), _p(hp.lr), c_dbl(hp.beta1), c_dbl(hp.beta2),
                             c_dbl(hp.eps), c_dbl(wd), C.c_int(hp.max_defer), C.c_int(mode))


def sgdm_deferred(w, b, counter, ids, g_compact, lr, mu, max_defer=15, mode=0):
    """Deferred momentum SGD (in place); mode 0 tables, mode 1 replay."""
    D, n = w.shape
    lr = np.full(6, lr, np.float64) if np.isscalar(lr) else np.asarray(lr, np.float64)
    ids = np.ascontiguousarray(ids, np.int32)
    gc = np.ascontiguousarray(g_compact, np.float64).reshape(D, ids.shape[0])
    assert counter.dtype == np.uint8
    lib().orc_sgdm_deferred(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(b), _p(counter), _p(ids), c_i64(ids.shape[0]),
                            _p(gc), _p(lr), c_dbl(mu), C.c_int(max_defer), C.c_int(mode))


def adamw_materialize(w, m, v, counter, t_done, hp: AdamHyper, wd, mode=0):
    D, n = w.shape
    wo, mo, vo = np.zeros_like(w), np.zeros_like(m), np.zeros_like(v)
    lib().orc_adamw_materialize(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(m), _p(v), _p(counter), C.c_int(t_done),
                                _p(hp.lr), c_dbl(hp.beta1), c_dbl(hp.beta2), c_dbl(hp.eps), c_dbl(wd),
                                C.c_int(hp.max_defer), C.c_int(mode), _p(wo), _p(mo), _p(vo))
    return wo, mo, vo


def sgdm_materialize(w, b, counter, lr, mu, max_defer=15, mode=0):
    D, n = w.shape
    lr = np.full(6, lr, np.float64) if np.isscalar(lr) else np.asarray(lr, np.float64)
    wo, bo = np.zeros_like(w), np.zeros_like(b)
    lib().orc_sgdm_materialize(c_i64(n), C.c_int(D), c_i64(n), _p(w), _p(b), _p(counter), _p(lr), c_dbl(mu),
                               C.c_int(max_defer), C.c_int(mode), _p(wo), _p(bo))
    return wo, bo


# ---------------------------------------------------------------------------- densification (§2.4 step 7)

def densify(w, m, v, counter, t_done, hp: AdamHyper, grad_accum, denom, extent, normals, grad_threshold=2e-4,
            percent_dense=0.01, min_opacity=0.005, mode=0, geo_eager=False):
    """Periodic densification (§2.4 step 7: clone or split Gaussians with large
    accumulated gradients, prune low-opacity ones) on a deferred-Adam state
    after t_done steps.  The paper names the step and defers to 3DGS; the rules
    are 3DGS's: g = grad_accum / denom (mean view-space gradient norm, 0 where
    never seen); g >= grad_threshold clones a Gaussian whose largest scale is at
    most percent_dense * extent and splits a larger one into two children
    (scales / 1.6, means mu + R(q) (s * z) for the standard normals
    normals[j] [3][n_split] passed in); then every Gaussian whose opacity is
    below min_opacity is pruned.  New Gaussians get zero moments.

    Deferred state: every decision reads the current (caught-up) values; a
    row that is copied or split is caught up first (counter 0); other rows keep
    their deferred w, m, v and counter.  Order of the result: survivors in
    their order, then clones, then the children of split 0, then of split 1 (3DGS's).
    Returns (w, m, v, counter)."""
    from scipy.spatial.transform import Rotation
    D, n = w.shape
    wc, mc, vc = adam_materialize(w, m, v, counter, t_done, hp, mode=mode, geo_eager=geo_eager)
    g = np.where(denom > 0, grad_accum / np.where(denom > 0, denom, 1), 0.0)
    smax = np.exp(wc[3:6]).max(axis=0)
    big = g >= grad_threshold
    clone = big & (smax <= percent_dense * extent)
    split = big & (smax > percent_dense * extent)
    wd_, md_, vd_, cd_ = w.copy(), m.copy(), v.copy(), counter.copy()
    aff = clone | split
    wd_[:, aff], md_[:, aff], vd_[:, aff], cd_[aff] = wc[:, aff], mc[:, aff], vc[:, aff], 0
    ids_s = np.nonzero(split)[0]
    q = wc[6:10, ids_s]                                            # (w, x, y, z)
    R = Rotation.from_quat(np.stack([q[1], q[2], q[3], q[0]], axis=1)).as_matrix() if len(ids_s) else np.zeros((0, 3, 3))
    s = np.exp(wc[3:6, ids_s])
    parts_w = [wd_[:, ~split], wc[:, clone]]
    cur_w = [wc[:, ~split], wc[:, clone]]                          # current values, for the prune decision
    for j in range(2):
        child = wc[:, ids_s].copy()
        child[0:3] += np.einsum("kab,bk->ak", R, s * normals[j])
        child[3:6] = np.log(s / 1.6)
        parts_w.append(child)
        cur_w.append(child)
    n_new = int(clone.sum()) + 2 * len(ids_s)
    W2 = np.concatenate(parts_w, axis=1)
    M2 = np.concatenate([md_[:, ~split], np.zeros((D, n_new))], axis=1)
    V2 = np.concatenate([vd_[:, ~split], np.zeros((D, n_new))], axis=1)
    C2 = np.concatenate([cd_[~split], np.zeros(n_new, np.uint8)])
    opac = 1.0 / (1.0 + np.exp(-np.concatenate(cur_w, axis=1)[10]))
    keep = opac >= min_opacity
    return (np.ascontiguousarray(W2[:, keep]), np.ascontiguousarray(M2[:, keep]),
            np.ascontiguousarray(V2[:, keep]), np.ascontiguousarray(C2[keep]))
