"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Discrete results (cull sets, key lists, counters) are
bit-exact except decisions whose FP64 margin is a tie at FP32 resolution;
images within 1e-5 absolute, gradients within 1e-4 relative (per parameter
group), optimizer state within FP32 rounding of the FP64 values."""
import math

import numpy as np
import pytest
import torch

from helpers import GROUPS, TIE_TOL, cam_f32, check_lists, f32, hp32, rel_group_error
from helpers import pixel_exclusions as _pixel_exclusions
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2509_15645_b300 as gs
    return gs


def make_ctx(gs, n, W, H, deg=3, tile=(16, 16), max_vis=None, max_keys=None, views=1, list_records=0):
    return gs.Context(max_gaussians=n, max_visible=max_vis or n, max_keys=max_keys or (64 * n + 4096),
                      max_width=W, max_height=H, tile=tile, max_views=views, max_sh_degree=deg,
                      list_records=list_records)


def _case(name):
    """(params float32 [D][n], camera, sh degree, tile)."""
    if name == "cube10k":
        c = scenes.cfg_small_step()
        return c["scene"], c["cams"][0], 0, (16, 16)
    if name == "cube_offaxis_sh3":
        P = scenes.uniform_cube_scene(6000, seed=3, sh_degree=3, log_scale_mean=-3.2)
        P[14:] *= 10.0
        cam = scenes.camera_lookat((0.9, -0.6, -2.4), (0.4, 0.3, 0.2), 96, 72, 70.0, up=(0, -1, 0))
        return P, cam, 3, (16, 16)
    if name == "ragged_tiles":
        P = scenes.uniform_cube_scene(1037, seed=4, sh_degree=1, log_scale_mean=-2.5)
        cam = scenes.camera_lookat((0.1, 0.2, -3.0), (0.0, 0.0, 0.0), 77, 45, 60.0, up=(0, -1, 0))
        return P, cam, 1, (16, 16)
    if name == "tile32x8":
        P = scenes.uniform_cube_scene(3000, seed=5, sh_degree=2, log_scale_mean=-3.0)
        cam = scenes.camera_lookat((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 80, 64, 60.0, up=(0, -1, 0))
        return P, cam, 2, (32, 8)
    if name == "tile8x4_ragged":
        # the benchmark's tile shape (one warp per tile), ragged in both directions
        P = scenes.uniform_cube_scene(3000, seed=6, sh_degree=3, log_scale_mean=-3.0)
        cam = scenes.camera_lookat((0.3, -0.2, -2.8), (0.0, 0.1, 0.0), 90, 70, 65.0, up=(0, -1, 0))
        return P, cam, 3, (8, 4)
    if name == "degenerate":
        c = scenes.cfg_diff_check(n=8000, width=96)
        return c["scene"], c["cams"][0], 3, (16, 16)
    if name == "needles":
        # long thin Gaussians at random orientations: a near-singular 2D
        # covariance (diagonal in the image) or a needle seen end-on, where the
        # FP32 covariance chain loses 10+ bits and the FP64 path takes over
        P = scenes.uniform_cube_scene(1200, seed=12, sh_degree=1, log_scale_mean=-3.0)
        P[3] = -0.8
        P[4:6] = -7.5
        cam = scenes.camera_lookat((0.2, -0.3, -3.2), (0.0, 0.0, 0.0), 96, 72, 60.0, up=(0, -1, 0))
        return P, cam, 1, (16, 16)
    raise KeyError(name)


CASES = ["cube10k", "cube_offaxis_sh3", "ragged_tiles", "tile32x8", "tile8x4_ragged", "degenerate"]


def _run_fwd(gs, orc, name):
    P, cam, deg, tile = _case(name)
    camf = cam_f32(cam)
    n = P.shape[1]
    ctx = make_ctx(gs, n, camf.width, camf.height, deg=3, tile=tile)
    scene = gs.GaussianScene(P, deg)
    ids, nv = ctx.cull(scene, camf)
    img = ctx.render_fwd(scene, camf, ids, nv)
    ctx.sync_status()
    nvis = int(nv.item())
    gids = ids[:nvis].cpu().numpy()
    r = orc.render(f32(P), deg, camf, tile)
    return dict(P=P, cam=camf, deg=deg, tile=tile, ctx=ctx, scene=scene, ids=ids, nv=nv, gids=gids,
                img=img.cpu().numpy().astype(np.float64), r=r)


@pytest.mark.parametrize("name", CASES)
def test_cull_parity(gs, orc, name):
    d = _run_fwd(gs, orc, name)
    sp = d["r"]["splats"]
    kept = np.nonzero(sp["keep"])[0]
    tie = sp["margin"] < TIE_TOL
    assert np.all(np.diff(d["gids"]) > 0), "ids must be ascending"
    diff = np.setxor1d(d["gids"], kept)
    assert np.all(tie[diff]), f"non-tie cull mismatches: {diff[~tie[diff]][:10]}"
    assert tie.sum() <= max(3, 0.01 * sp.shape[0])
    assert len(kept) > 0


# The GPU's list filter (k_lists.cu) is the oracle's reach rule evaluated in
# FP32 and made conservative by a stated slack: the square widened by 1e-3
# pixel and the floor lowered by 0.1%.  A pair the oracle drops may therefore
# appear on the GPU only if its FP64 reach with twice that slack passes.
REACH_EXT, REACH_FLOOR = 2e-3, (1.0 / 255.0) * 0.998


@pytest.mark.parametrize("name", CASES)
def test_key_lists_parity(gs, orc, name):
    d = _run_fwd(gs, orc, name)
    r = d["r"]
    tx, ty = (d["cam"].width + d["tile"][0] - 1) // d["tile"][0], (d["cam"].height + d["tile"][1] - 1) // d["tile"][1]
    keys, vals, ranges = d["ctx"].render_lists(tx * ty)
    keys = keys.cpu().numpy().astype(np.int64)
    vals = vals.cpu().numpy().astype(np.int64)
    gpu_gid = d["gids"][vals]
    sp = r["splats"]
    # Gaussians whose cull or integer radius is a tie at FP32 resolution
    exclude = np.nonzero((sp["margin"] < TIE_TOL) | (sp["radius_margin"] < TIE_TOL))[0]
    dbits = sp["depth"].astype(np.float32).view(np.uint32)
    ot, og = r["key_tile"].astype(np.int64), r["key_gid"].astype(np.int64)
    o_pairs = set(zip(ot.tolist(), og.tolist()))
    g_pairs = set(zip(keys.tolist(), gpu_gid.tolist()))
    missing = [(t, g) for (t, g) in o_pairs - g_pairs if g not in set(exclude.tolist())]
    assert not missing, f"pairs of the oracle's lists missing on the GPU: {missing[:8]}"
    extra = np.array([(t, g) for (t, g) in g_pairs - o_pairs if g not in set(exclude.tolist())], np.int64)
    n_extra = len(extra)
    if n_extra:
        slack = orc.tile_reach(sp, r["cam"], extra[:, 1], extra[:, 0], ext=REACH_EXT)
        assert np.all(slack >= REACH_FLOOR), extra[slack < REACH_FLOOR][:8]
    # the sequences agree once the tie Gaussians and the slack pairs are dropped
    drop_extra = set(map(tuple, extra.tolist())) if n_extra else set()
    keep_g = np.array([(t, g) not in drop_extra for t, g in zip(keys.tolist(), gpu_gid.tolist())], bool)
    swaps = check_lists(keys[keep_g], gpu_gid[keep_g], ot, og, dbits, exclude)
    assert swaps <= 4
    assert n_extra <= 1e-3 * len(ot) + 2, (n_extra, len(ot))
    print(f"{name}: {len(ot)} keys, {n_extra} slack pairs, {len(exclude)} tie Gaussians, {swaps} depth-tie swaps")
    # ranges delimit each tile's run
    rg = ranges.cpu().numpy().astype(np.int64)
    for t in range(tx * ty):
        b, e = rg[t]
        assert np.all(keys[b:e] == t)
        assert e - b == np.count_nonzero(keys == t)


@pytest.mark.parametrize("name", CASES)
def test_render_forward_parity(gs, orc, name):
    d = _run_fwd(gs, orc, name)
    ref = d["r"]["image"]
    ex = _pixel_exclusions(d["r"], d["gids"])
    err = np.abs(d["img"] - ref)
    ok = ~ex[None, :, :].repeat(3, 0)
    assert ex.mean() < 0.03, f"too many tie pixels: {ex.mean()}"
    assert err[ok].max() <= 1e-5, (err[ok].max(), np.unravel_index(np.argmax(np.where(ok, err, 0)), err.shape))
    assert ref.max() > 0.05
    n_fp64 = int(d["ctx"].counters()[6].item())
    assert n_fp64 <= 0.01 * len(d["gids"]), n_fp64        # rare on moderately anisotropic scenes


def test_fp64_covariance_needles(gs, orc):
    """Long thin Gaussians (one axis 0.45, two 5.5e-4) at random orientations:
    the FP32 covariance chain would leave a relative conic error of about
    u * (a + c) * tr(Sigma3) * |T|^2 / det, here up to 1.5e-4, so every one of
    them goes through the FP64 chain, whose conic must agree with the FP64
    oracle to FP32 rounding.  The image and the gradients are then bounded by
    what FP32 compositing allows: sigma at a pixel sums terms of up to
    sigma_abs = (|A| + 2|B| + |C|) r^2 / 2 that cancel, so alpha and its
    derivatives carry a relative error of up to about 8 u sigma_abs."""
    d = _run_fwd(gs, orc, "needles")
    r, ctx, gids = d["r"], d["ctx"], d["gids"]
    sp = r["splats"]
    geom, conic = ctx.render_splats()
    geom = geom.cpu().numpy().astype(np.float64)
    conic = conic.cpu().numpy().astype(np.float64)
    n_fp64 = int(ctx.counters()[6].item())
    kept = sp["keep"][gids] == 1
    assert n_fp64 >= 0.9 * len(gids) and kept.sum() > 0.9 * len(gids), (n_fp64, len(gids))
    ref_c = sp["conic"][gids][kept]
    scale = np.abs(ref_c[:, 0]) + np.abs(ref_c[:, 2])
    cerr = np.abs(conic[kept, :3] - ref_c) / scale[:, None]
    assert cerr.max() <= 4e-7, cerr.max()
    assert np.abs(geom[kept, :2] - sp["mean2d"][gids][kept]).max() <= 1e-4
    tie = sp["radius_margin"][gids][kept] < TIE_TOL
    assert np.all((geom[kept, 2] == sp["radius"][gids][kept]) | tie)
    # image and gradients within the FP32-compositing bound
    con, rad = sp["conic"][sp["keep"] == 1], sp["radius"][sp["keep"] == 1]
    sabs = 0.5 * (np.abs(con[:, 0]) + 2 * np.abs(con[:, 1]) + np.abs(con[:, 2])) * rad ** 2
    bound = 8 * 2.0 ** -24 * sabs.max()
    ex = _pixel_exclusions(r, gids)
    assert ex.mean() < 0.1, ex.mean()
    err = np.abs(d["img"] - r["image"])[:, ~ex]
    assert err.max() <= bound, (err.max(), bound)
    P, cam, deg, tile = d["P"], d["cam"], d["deg"], d["tile"]
    target = _target(orc, P, cam, deg, tile, seed=11)
    _, dimg = orc.loss_l1(r["image"], target)
    g_ref, _ = orc.backward(f32(P), deg, r["cam"], r["splats"], r["key_gid"], r["ranges"], dimg)
    gc = ctx.render_bwd(torch.as_tensor(dimg, dtype=torch.float32, device="cuda"), P.shape[0])
    full = ctx.grad_scatter(d["scene"], d["ids"], d["nv"], gc)
    ctx.sync_status()
    g_gpu = full[:, :P.shape[1]].cpu().numpy().astype(np.float64)
    errs = {k: rel_group_error(g_gpu, g_ref, s) for k, s in GROUPS.items() if g_ref[s].size}
    assert max(errs.values()) <= bound, (errs, bound)


def _target(orc, P_like, cam, deg, tile, seed):
    T = scenes.uniform_cube_scene(P_like.shape[1], seed=seed, sh_degree=deg)
    return orc.render(f32(T), deg, cam, tile)["image"]


@pytest.mark.parametrize("name", CASES)
def test_render_backward_parity(gs, orc, name):
    d = _run_fwd(gs, orc, name)
    P, cam, deg, tile = d["P"], d["cam"], d["deg"], d["tile"]
    target = _target(orc, P, cam, deg, tile, seed=11)
    r = d["r"]
    loss, dimg = orc.loss_l1(r["image"], target)
    g_ref, _ = orc.backward(f32(P), deg, r["cam"], r["splats"], r["key_gid"], r["ranges"], dimg)
    D = P.shape[0]
    dimg_t = torch.as_tensor(dimg, dtype=torch.float32, device="cuda")
    gc = d["ctx"].render_bwd(dimg_t, D)
    full = d["ctx"].grad_scatter(d["scene"], d["ids"], d["nv"], gc)
    d["ctx"].sync_status()
    g_gpu = full[:, :P.shape[1]].cpu().numpy().astype(np.float64)
    errs = {k: rel_group_error(g_gpu, g_ref, s) for k, s in GROUPS.items() if g_ref[s].size}
    assert max(errs.values()) <= 1e-4, errs


@pytest.mark.parametrize("name,tile", [("cube_offaxis_sh3", (16, 16)), ("ragged_tiles", (16, 16)),
                                       ("tile32x8", (32, 8)), ("cube10k", (8, 8)), ("cube10k", (16, 8)),
                                       ("cube10k", (64, 4)), ("cube_offaxis_sh3", (8, 4)), ("ragged_tiles", (4, 8))])
def test_raster_variants_agree(gs, orc, name, tile):
    """Every rasterizer variant (pixels per thread, batch) the tile shape allows
    renders the same image bit for bit, and its gradients match the oracle."""
    P, cam, deg, _ = _case(name)
    camf = cam_f32(cam)
    n, D = P.shape[1], P.shape[0]
    ctx = make_ctx(gs, n, camf.width, camf.height, deg=3, tile=tile, list_records=1)
    scene = gs.GaussianScene(P, deg)
    ids, nv = ctx.cull(scene, camf)
    r = orc.render(f32(P), deg, camf, tile)
    dimg = np.random.default_rng(2).normal(size=r["image"].shape)
    g_ref, _ = orc.backward(f32(P), deg, r["cam"], r["splats"], r["key_gid"], r["ranges"], dimg)
    dimg_t = torch.as_tensor(dimg, dtype=torch.float32, device="cuda")
    from paper_2509_15645_b300 import _lib
    images, tried = [], 0
    for v in range(_lib.RASTER_VARIANTS):
        try:
            ctx.set_raster_variant(v)
        except Exception:
            continue
        tried += 1
        img = ctx.render_fwd(scene, camf, ids, nv)
        gc = ctx.render_bwd(dimg_t, D)
        full = ctx.grad_scatter(scene, ids, nv, gc)
        ctx.sync_status()
        images.append(img.cpu().numpy())
        g_gpu = full[:, :n].cpu().numpy().astype(np.float64)
        errs = {k: rel_group_error(g_gpu, g_ref, sl) for k, sl in GROUPS.items() if g_ref[sl].size}
        assert max(errs.values()) <= 1e-4, (v, errs)
    assert tried >= 2
    if tile[0] * tile[1] == 32:
        assert tried >= 5                    # the warp-tile variants 6-9 among them
    for im in images[1:]:
        np.testing.assert_array_equal(im, images[0])
    (vf, vb), ms_f, ms_b = ctx.autotune(scene, camf)
    assert ms_f[vf] is not None and ms_f[vf] == min(t for t in ms_f if t is not None)
    assert ms_b[vb] is not None and ms_b[vb] == min(t for t in ms_b if t is not None)


def test_raster_pair_counts(gs, orc):
    """The backward's work counts: contributing pairs equal the oracle's
    contributor counts summed over pixels (ties aside)."""
    P, cam, deg, tile = _case("cube_offaxis_sh3")
    camf = cam_f32(cam)
    ctx = make_ctx(gs, P.shape[1], camf.width, camf.height, deg=3, tile=tile)
    scene = gs.GaussianScene(P, deg)
    n_sq, n_on, n_empty = ctx.raster_pair_counts(scene, camf)
    r = orc.render(f32(P), deg, camf, tile)
    ex = r["margin"] < TIE_TOL
    ref = int(r["n_contrib"].sum())
    assert abs(n_on - ref) <= 2 * int(ex.sum()) + 2, (n_on, ref)
    assert n_sq >= n_on > 0
    assert n_empty == 0                        # counted on 32-pixel tiles only
    # 8x4 tiles: keys whose tile takes the splat at no pixel, fewer than the keys
    P2, cam2, deg2, tile2 = _case("tile8x4_ragged")
    cam2 = cam_f32(cam2)
    ctx2 = make_ctx(gs, P2.shape[1], cam2.width, cam2.height, deg=deg2, tile=tile2)
    s2 = gs.GaussianScene(P2, deg2)
    n_sq2, n_on2, n_empty2 = ctx2.raster_pair_counts(s2, cam2)
    keys = int(orc.render(f32(P2), deg2, cam2, tile2)["key_gid"].shape[0])
    assert 0 < n_empty2 < keys and n_on2 > 0, (n_empty2, keys)


def test_loss_l1_kernel(gs):
    ctx = make_ctx(gs, 64, 40, 30)
    rng = np.random.default_rng(0)
    a = rng.random((3, 30, 40)).astype(np.float32)
    b = rng.random((3, 30, 40)).astype(np.float32)
    b[1, 2, 3] = a[1, 2, 3]
    ta, tb = torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda")
    loss, dimg = ctx.loss_l1(ta, tb)
    ctx.sync_status()
    ref = np.mean(np.abs(a.astype(np.float64) - b))
    assert abs(loss.item() - ref) <= 1e-6 * ref
    np.testing.assert_array_equal(dimg.cpu().numpy(), (np.sign(a - b) / a.size).astype(np.float32))


# ---------------------------------------------------------------------------- Adam

def _adam_state(rng, D, n, t):
    w = rng.normal(size=(D, n)).astype(np.float32)
    m = (rng.normal(size=(D, n)) * 1e-3).astype(np.float32)
    v = rng.uniform(1e-8, 1e-6, size=(D, n)).astype(np.float32)
    cnt = rng.integers(0, min(16, t), n).astype(np.uint8)
    return w, m, v, cnt


@pytest.mark.parametrize("mode", ["deferred", "eager"])
@pytest.mark.parametrize("n,t", [(1000, 40), (4099, 3), (70001, 500)])
def test_adam_step_parity(gs, orc, mode, n, t):
    rng = np.random.default_rng(n + t)
    deg, D = 3, 59
    w, m, v, cnt = _adam_state(rng, D, n, t)
    lr = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4]
    ids = np.sort(rng.choice(n, n // 5, replace=False)).astype(np.int32)
    gc = (rng.normal(size=(D, ids.size)) * 1e-3).astype(np.float32)
    scene = gs.GaussianScene(w, deg)
    scene.m[:, :n] = torch.as_tensor(m, device="cuda")
    scene.v[:, :n] = torch.as_tensor(v, device="cuda")
    scene.counter[:n] = torch.as_tensor(cnt, device="cuda")
    scene.step = t - 1
    ctx = make_ctx(gs, n, 64, 64)
    adam = gs.adam_struct(lr=lr, eps=1e-15, mode=0 if mode == "deferred" else 2)
    ids_t = torch.as_tensor(ids, device="cuda")
    nv = torch.tensor([ids.size], dtype=torch.int32, device="cuda")
    gct = torch.zeros(D, ctx.max_visible, dtype=torch.float32, device="cuda")
    gct[:, :ids.size] = torch.as_tensor(gc, device="cuda")
    ctx.adam_deferred(scene, ids_t, nv, gct, adam)
    ctx.sync_status()
    hp = hp32(orc, lr=lr, eps=1e-15)
    W, M, V, Cn = f32(w), f32(m), f32(v), cnt.copy()
    if mode == "deferred":
        orc.adam_deferred(W, M, V, Cn, ids, f32(gc), t, hp, mode=0)
    else:
        g = np.zeros((D, n))
        g[:, ids] = f32(gc)
        orc.adam_eager(W, M, V, g, t, hp)
    gw = scene.w[:, :n].cpu().numpy().astype(np.float64)
    gm = scene.m[:, :n].cpu().numpy().astype(np.float64)
    gv = scene.v[:, :n].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(scene.counter[:n].cpu().numpy(), Cn)
    assert scene.step == t
    # FP32 error bounds: every term of each update rounds with relative error u
    u = 2.0 ** -24
    g = np.zeros((D, n))
    g[:, ids] = f32(gc)
    upd = np.zeros(n, bool)
    upd[ids] = True
    if mode == "deferred":
        upd |= cnt >= 15
        dly = np.where(upd, cnt, 0).astype(int)
    else:
        upd[:] = True
        dly = np.zeros(n, int)
    m0, v0, w0 = f32(m), f32(v), f32(w)
    b1p, b2p = hp.beta1 ** (dly + 1), hp.beta2 ** (dly + 1)
    bm = 8 * u * (b1p * np.abs(m0) + (1 - hp.beta1) * np.abs(g)) + 1e-30
    bv = 8 * u * (b2p * v0 + (1 - hp.beta2) * g * g) + 1e-38
    restore = np.zeros((D, n))
    for grp, rows in enumerate([slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, D)]):
        pl, _, _ = orc.adam_lut(t, hp.lr[grp], hp)
        pl = np.nan_to_num(pl)
        restore[rows] = pl[dly] * np.abs(m0[rows]) / np.sqrt(v0[rows])
    bw = 16 * u * (np.abs(w0) + restore + np.abs(W - w0)) + 1e-30
    for name, a, b, bound in (("m", gm, M, bm), ("v", gv, V, bv), ("w", gw, W, bw)):
        err = np.abs(a - b)
        assert np.all(err[:, upd] <= bound[:, upd]), (name, np.max(err / bound))
        np.testing.assert_array_equal(a[:, ~upd], b[:, ~upd])   # untouched


@pytest.mark.parametrize("opt", ["adamw", "sgdm"])
@pytest.mark.parametrize("mode", ["deferred", "eager"])
@pytest.mark.parametrize("n,t", [(1000, 40), (70001, 500)])
def test_optimizer_variant_step_parity(gs, orc, opt, mode, n, t):
    """Deferred AdamW (decoupled decay, restore w <- decay[d] w - wlut[d] m /
    (sqrt(v) + eps)) and deferred momentum SGD (restore w <- w - slut[d] b, b
    <- mu^(d+1) b + g) against the oracle's steps of the same optimizer from the
    same stored state, within FP32 rounding of each update term; counters
    bit-exact; Gaussians outside the update set untouched."""
    from paper_2509_15645_b300 import _lib
    rng = np.random.default_rng(n + t + (7 if opt == "sgdm" else 0))
    deg, D = 3, 59
    w, m, v, cnt = _adam_state(rng, D, n, t)
    lr = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4]
    wd, mu = 0.05, 0.9
    ids = np.sort(rng.choice(n, n // 5, replace=False)).astype(np.int32)
    gc = (rng.normal(size=(D, ids.size)) * 1e-3).astype(np.float32)
    scene = gs.GaussianScene(w, deg)
    scene.m[:, :n] = torch.as_tensor(m, device="cuda")
    scene.v[:, :n] = torch.as_tensor(v, device="cuda")
    scene.counter[:n] = torch.as_tensor(cnt, device="cuda")
    scene.step = t - 1
    ctx = make_ctx(gs, n, 64, 64)
    kind = _lib.GS_OPT_ADAMW if opt == "adamw" else _lib.GS_OPT_SGDM
    adam = gs.adam_struct(lr=lr, eps=1e-15, beta1=mu if opt == "sgdm" else 0.9, mode=0 if mode == "deferred" else 2,
                          optimizer=kind, weight_decay=wd)
    ctx.refresh_rdir(scene, adam)              # m, v were set directly
    ids_t = torch.as_tensor(ids, device="cuda")
    nv = torch.tensor([ids.size], dtype=torch.int32, device="cuda")
    gct = torch.zeros(D, ctx.max_visible, dtype=torch.float32, device="cuda")
    gct[:, :ids.size] = torch.as_tensor(gc, device="cuda")
    ctx.adam_deferred(scene, ids_t, nv, gct, adam)
    ctx.sync_status()
    hp = hp32(orc, lr=lr, eps=1e-15)
    lr32 = hp.lr
    W, M, V, Cn = f32(w), f32(m), f32(v), cnt.copy()
    g = np.zeros((D, n))
    g[:, ids] = f32(gc)
    wd32, mu32 = float(np.float32(wd)), float(np.float32(mu))
    if opt == "adamw" and mode == "deferred":
        orc.adamw_deferred(W, M, V, Cn, ids, f32(gc), t, hp, wd32, mode=0)
    elif opt == "adamw":
        orc.adamw_eager(W, M, V, g, t, hp, wd32)
    elif mode == "deferred":
        orc.sgdm_deferred(W, M, Cn, ids, f32(gc), lr32, mu32, max_defer=15, mode=0)
    else:
        orc.sgdm_eager(W, M, g, lr32, mu32)
    gw = scene.w[:, :n].cpu().numpy().astype(np.float64)
    gm = scene.m[:, :n].cpu().numpy().astype(np.float64)
    gv = scene.v[:, :n].cpu().numpy().astype(np.float64)
    if mode == "deferred":
        np.testing.assert_array_equal(scene.counter[:n].cpu().numpy(), Cn)
    u = 2.0 ** -24
    upd = np.zeros(n, bool)
    upd[ids] = True
    if mode == "deferred":
        upd |= cnt >= 15
        dly = np.where(upd, cnt, 0).astype(int)
    else:
        upd[:] = True
        dly = np.zeros(n, int)
    m0, v0, w0 = f32(m), f32(v), f32(w)
    restore = np.zeros((D, n))
    for grp, rows in enumerate([slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, D)]):
        if opt == "adamw":
            wl, _ = orc.adamw_lut(t, lr32[grp], hp, wd32)
            restore[rows] = np.nan_to_num(wl)[dly] * np.abs(m0[rows]) / np.sqrt(v0[rows])
        else:
            sl, _ = orc.sgdm_lut(lr32[grp], mu32, 15)
            restore[rows] = sl[dly] * np.abs(m0[rows]) + lr32[grp] * np.abs(M[rows])
    if opt == "adamw":
        b1p, b2p = hp.beta1 ** (dly + 1), hp.beta2 ** (dly + 1)
        bm = 8 * u * (b1p * np.abs(m0) + (1 - hp.beta1) * np.abs(g)) + 1e-30
        bv = 8 * u * (b2p * v0 + (1 - hp.beta2) * g * g) + 1e-38
        checks = (("m", gm, M, bm), ("v", gv, V, bv))
    else:
        bm = 8 * u * (mu32 ** (dly + 1) * np.abs(m0) + np.abs(g)) + 1e-30
        checks = (("m", gm, M, bm),)
        np.testing.assert_array_equal(gv, v0)          # momentum SGD keeps no v: never written
    bw = 16 * u * (np.abs(w0) + restore + np.abs(W - w0)) + 1e-30
    for name, a, b, bound in checks + (("w", gw, W, bw),):
        err = np.abs(a - b)
        assert np.all(err[:, upd] <= bound[:, upd]), (name, np.max(err / bound))
        np.testing.assert_array_equal(a[:, ~upd], b[:, ~upd])   # untouched


def test_materialize_parity(gs, orc):
    rng = np.random.default_rng(5)
    n, D, t_done = 5000, 14, 30
    w, m, v, cnt = _adam_state(rng, D, n, t_done + 1)
    scene = gs.GaussianScene(w, 0)
    scene.m[:, :n] = torch.as_tensor(m, device="cuda")
    scene.v[:, :n] = torch.as_tensor(v, device="cuda")
    scene.counter[:n] = torch.as_tensor(cnt, device="cuda")
    scene.step = t_done
    ctx = make_ctx(gs, n, 64, 64, deg=0)
    adam = gs.adam_struct(lr=1e-3, eps=1e-15)
    wo, mo, vo = ctx.materialize(scene, adam)
    ctx.sync_status()
    hp = hp32(orc, lr=1e-3, eps=1e-15)
    W, M, V = orc.adam_materialize(f32(w), f32(m), f32(v), cnt, t_done, hp, mode=0)
    u = 2.0 ** -24
    np.testing.assert_allclose(mo[:, :n].cpu().numpy(), M, rtol=8 * u, atol=0)
    np.testing.assert_allclose(vo[:, :n].cpu().numpy(), V, rtol=8 * u, atol=0)
    gw = wo[:, :n].cpu().numpy().astype(np.float64)
    bound = 16 * u * (np.abs(f32(w)) + np.abs(W - f32(w)))
    assert np.all(np.abs(gw - W) <= bound + 1e-30), np.max(np.abs(gw - W) / (bound + 1e-30))


@pytest.mark.parametrize("bf16", [False, True])
def test_restore_directions(gs, bf16):
    """The kept restore directions equal m / (sqrt(v) + eps) (rounded to the
    plane's type: fp32 geometry planes, SH planes in the SH type) after a
    refresh and after optimizer steps, and restoring through them gives the
    same cull and (fp32 form) the same image as recomputing from m and v."""
    from paper_2509_15645_b300 import _lib
    rng = np.random.default_rng(12)
    n, deg = 6000, 1
    P = scenes.uniform_cube_scene(n, seed=12, sh_degree=deg, log_scale_mean=-3.0)
    scene = gs.GaussianScene(P, deg, precision=_lib.GS_BF16_SH_MOM if bf16 else _lib.GS_FP32)
    D = scene.D
    mdt = scene.m.dtype
    scene.m[:, :n] = torch.as_tensor(rng.normal(size=(D, n)) * 1e-2, dtype=torch.float32, device="cuda").to(mdt)
    scene.v[:, :n] = torch.as_tensor(rng.uniform(1e-8, 1e-5, (D, n)), dtype=torch.float32, device="cuda").to(mdt)
    scene.counter[:n] = torch.as_tensor(rng.integers(0, 16, n), dtype=torch.uint8, device="cuda")
    scene.step = 30
    adam = gs.adam_struct(lr=1e-2, eps=1e-15)
    cam = scenes.camera_lookat((0.3, -0.2, -3.0), (0.0, 0.0, 0.0), 96, 64, 60.0, up=(0, -1, 0))
    ctx = make_ctx(gs, n, 96, 64, deg=deg)
    ctx.refresh_rdir(scene, adam)
    eps32 = np.float32(1e-15)
    u32 = 2.0 ** -24                                    # the direction uses a 2-ulp divide

    def check(sc):
        m = sc.m[:, :n].float().cpu().numpy()
        v = sc.v[:, :n].float().cpu().numpy()
        ref = m / (np.sqrt(v) + eps32)
        np.testing.assert_allclose(sc.rdir_geo[:, :n].cpu().numpy(), ref[:11], rtol=6 * u32, atol=0)

    check(scene)
    ids_a, nv_a = ctx.cull(scene, cam, adam)
    img_a = ctx.render_fwd(scene, cam, ids_a, nv_a, adam)
    kept = scene.rdir_geo
    scene.rdir_geo = None                               # recompute from m and v
    ids_b, nv_b = ctx.cull(scene, cam, adam)
    img_b = ctx.render_fwd(scene, cam, ids_b, nv_b, adam)
    ctx.sync_status()
    scene.rdir_geo = kept
    assert nv_a.item() == nv_b.item() > 0
    assert torch.equal(ids_a[:nv_a.item()], ids_b[:nv_b.item()])
    assert torch.equal(img_a, img_b)     # a stored direction and a recomputed one restore bit for bit
    gc = torch.as_tensor(rng.normal(size=(D, ctx.max_visible)) * 1e-3, dtype=torch.float32, device="cuda")
    for _ in range(3):
        ctx.adam_deferred(scene, ids_a, nv_a, gc, adam)
    ctx.sync_status()
    check(scene)


def test_bf16_stochastic_rounding_keeps_decay(gs):
    """With zero gradients each eager step multiplies v by 0.999, which is
    below half a bf16 ulp: round-to-nearest rounds it back to v forever, while
    stochastic rounding decays v by 0.999 per step on average."""
    from paper_2509_15645_b300 import _lib
    n, deg, steps = 200_000, 0, 60
    rng = np.random.default_rng(4)
    P = scenes.uniform_cube_scene(n, seed=4, sh_degree=deg)
    ctx = make_ctx(gs, n, 32, 32, deg=deg)
    out = {}
    for prec in (_lib.GS_BF16_SH_MOM_RN, _lib.GS_BF16_SH_MOM):
        scene = gs.GaussianScene(P, deg, precision=prec)
        v0 = torch.as_tensor(rng.uniform(1.0, 2.0, (scene.D, n)), dtype=torch.float32, device="cuda")
        scene.v[:, :n] = v0.to(torch.bfloat16)
        v0 = scene.v[:, :n].float().clone()
        scene.m.zero_()
        ctx.refresh_rdir(scene, gs.adam_struct())
        ids = torch.zeros(1, dtype=torch.int32, device="cuda")
        nv = torch.zeros(1, dtype=torch.int32, device="cuda")
        gc = torch.zeros(scene.D, 8, device="cuda")
        for _ in range(steps):
            ctx.adam_deferred(scene, ids, nv, gc, gs.adam_struct(mode=_lib.GS_ADAM_EAGER, seed=7))
        ctx.sync_status()
        out[prec] = (scene.v[:, :n].float() / v0).mean().item()
    assert out[_lib.GS_BF16_SH_MOM_RN] == 1.0
    assert abs(out[_lib.GS_BF16_SH_MOM] - 0.999 ** steps) < 2e-4, out


def test_bf16_form_step_parity(gs, orc):
    """A whole step of the precision form (bf16 SH coefficients and moments,
    fp32 geometry and compositing, stochastic rounding of the stores) against
    the FP64 oracle step from the same stored state, three steps in a row.  The
    bf16 stores may differ from the exact values by less than one bf16 ulp
    (2^-7 relative); everything held in fp32 keeps the FP32 bounds."""
    from paper_2509_15645_b300 import _lib
    c = scenes.cfg_small_step()
    deg, tile = 3, (16, 16)
    P = scenes.uniform_cube_scene(c["scene"].shape[1], seed=8, sh_degree=deg, log_scale_mean=-2.8)
    cam = cam_f32(c["cams"][0])
    n, D = P.shape[1], P.shape[0]
    target = orc.render(f32(scenes.uniform_cube_scene(n, seed=9, sh_degree=deg, log_scale_mean=-2.8)), deg, cam,
                        tile)["image"]
    tgt = torch.as_tensor(target, dtype=torch.float32, device="cuda")
    scene = gs.GaussianScene(P, deg, precision=_lib.GS_BF16_SH_MOM)
    ctx = make_ctx(gs, n, cam.width, cam.height, deg=deg)
    lr = 1e-3
    adam = gs.adam_struct(lr=lr, eps=1e-15, seed=3)
    hp = hp32(orc, lr=lr, eps=1e-15)
    ub = 2.0 ** -7
    for t in (1, 2, 3):
        W = scene.params().cpu().numpy().astype(np.float64)
        M = scene.m[:, :n].float().cpu().numpy().astype(np.float64)
        V = scene.v[:, :n].float().cpu().numpy().astype(np.float64)
        Cn = scene.counter[:n].cpu().numpy().copy()
        W0 = W.copy()
        Wcur, _, _ = orc.adam_materialize(W, M, V, Cn, t - 1, hp)
        rr = orc.render_loss_backward(Wcur, deg, cam, target, tile)
        loss = ctx.step(scene, [cam], [tgt], adam)
        ctx.sync_status()
        assert abs(loss.item() - rr["loss"]) <= 1e-5 * rr["loss"] + 1e-7, (t, loss.item(), rr["loss"])
        # the gradients the step used, against the oracle's; then the oracle's
        # step fed those gradients, so the comparison is of the update alone
        sid, sg = ctx.step_gradients(D)
        sid = sid.cpu().numpy().astype(np.int32)
        g_step = sg.cpu().numpy().astype(np.float64)
        g_full = np.zeros((D, n))
        g_full[:, sid] = g_step
        for k, s in GROUPS.items():
            assert rel_group_error(g_full, rr["grad"], s) <= 1e-4, (t, k)
        orc.adam_deferred(W, M, V, Cn, sid, g_step, t, hp)
        np.testing.assert_array_equal(scene.counter[:n].cpu().numpy(), Cn)
        gw = scene.params().cpu().numpy().astype(np.float64)
        gm = scene.m[:, :n].float().cpu().numpy().astype(np.float64)
        gv = scene.v[:, :n].float().cpu().numpy().astype(np.float64)
        for k, s in GROUPS.items():
            if not M[s].size:
                continue
            scale_m, scale_v = np.abs(M[s]).max(), np.abs(V[s]).max()
            assert np.all(np.abs(gm[s] - M[s]) <= ub * np.abs(M[s]) + 2e-4 * scale_m), (t, k, "m")
            assert np.all(np.abs(gv[s] - V[s]) <= ub * np.abs(V[s]) + 4e-4 * scale_v), (t, k, "v")
        # geometry (fp32): the FP32 form's bound; SH (bf16): one ulp of the
        # stored value plus a 2^-6 relative error of the step lr * m/sqrt(v)
        gerr = np.abs(gw[:11] - W[:11])
        assert np.all(gerr <= 2e-3 * lr + 1e-6), (t, np.max(gerr))
        err = np.abs(gw[11:] - W[11:])
        bound = ub * np.abs(W[11:]) + 2 * ub * lr * (t + 1) + 1e-7
        assert np.all(err <= bound), (t, np.max(err / bound))
        moved = np.abs(W[11:] - W0[11:]) > 0
        assert moved.mean() > 0.1                      # the steps did update SH coefficients


def test_deferred_trajectory_tracks_eager(gs, orc):
    """Many GPU steps of deferred Adam, materialised, against the FP64 eager
    trajectory on the same gradients (the paper's claim of identical training
    up to the eps approximation, here at FP32)."""
    rng = np.random.default_rng(9)
    n, D, steps = 3000, 14, 60
    w0 = rng.normal(size=(D, n)).astype(np.float32)
    scene = gs.GaussianScene(w0, 0)
    ctx = make_ctx(gs, n, 64, 64, deg=0)
    adam = gs.adam_struct(lr=1e-3, eps=1e-15)
    hp = hp32(orc, lr=1e-3, eps=1e-15)
    We, Me, Ve = f32(w0), np.zeros((D, n)), np.zeros((D, n))
    for t in range(1, steps + 1):
        c = rng.integers(0, n)
        ids = np.arange(max(0, c - 300), min(n, c + 300), dtype=np.int32)
        gc = (rng.normal(size=(D, ids.size)) * 1e-2).astype(np.float32)
        gct = torch.zeros(D, ctx.max_visible, device="cuda")
        gct[:, :ids.size] = torch.as_tensor(gc, device="cuda")
        ctx.adam_deferred(scene, torch.as_tensor(ids, device="cuda"),
                          torch.tensor([ids.size], dtype=torch.int32, device="cuda"), gct, adam)
        g = np.zeros((D, n))
        g[:, ids] = f32(gc)
        orc.adam_eager(We, Me, Ve, g, t, hp)
    ctx.sync_status()
    wo, mo, vo = ctx.materialize(scene, adam)
    np.testing.assert_allclose(wo[:, :n].cpu().numpy(), We, rtol=0, atol=2e-5)
    np.testing.assert_allclose(mo[:, :n].cpu().numpy(), Me, rtol=1e-4, atol=1e-9)


# ---------------------------------------------------------------------------- whole step

def test_step_parity(gs, orc):
    """gs_step (CUDA graph: cull -> render -> L1 -> backward -> deferred Adam)
    against the oracle pipeline from the same state, twice in a row."""
    c = scenes.cfg_small_step()
    P, cam, deg, tile = c["scene"], cam_f32(c["cams"][0]), 0, (16, 16)
    n, D = P.shape[1], P.shape[0]
    target = orc.render(f32(c["target_scene"]), 0, cam, tile)["image"]
    scene = gs.GaussianScene(P, deg)
    ctx = make_ctx(gs, n, cam.width, cam.height, deg=0)
    adam = gs.adam_struct(lr=1e-3, eps=1e-15)
    hp = hp32(orc, lr=1e-3, eps=1e-15)
    tgt = torch.as_tensor(target, dtype=torch.float32, device="cuda")
    W, M, V, Cn = f32(P), np.zeros((D, n)), np.zeros((D, n)), np.zeros(n, np.uint8)
    for t in (1, 2):
        # oracle from the GPU's current state (one-step parity)
        W = scene.w[:, :n].cpu().numpy().astype(np.float64)
        M = scene.m[:, :n].cpu().numpy().astype(np.float64)
        V = scene.v[:, :n].cpu().numpy().astype(np.float64)
        Cn = scene.counter[:n].cpu().numpy().copy()
        Wcur, _, _ = orc.adam_materialize(W, M, V, Cn, t - 1, hp)   # current params for the render
        rr = orc.render_loss_backward(Wcur, deg, cam, target, tile)
        loss = ctx.step(scene, [cam], [tgt], adam)
        ctx.sync_status()
        assert abs(loss.item() - rr["loss"]) <= 1e-5 * rr["loss"] + 1e-7
        # the gradients the step used against the oracle's (per group), then
        # the oracle's step fed those gradients: the update alone, every entry
        # within FP32 rounding (no entry is left to the sign of a gradient)
        sid, sg = ctx.step_gradients(D)
        sid = sid.cpu().numpy().astype(np.int32)
        g_step = sg.cpu().numpy().astype(np.float64)
        kept = np.nonzero(rr["splats"]["keep"])[0].astype(np.int32)
        np.testing.assert_array_equal(sid, kept)
        g_full = np.zeros((D, n))
        g_full[:, sid] = g_step
        for k, s in GROUPS.items():
            if M[s].size:
                assert rel_group_error(g_full, rr["grad"], s) <= 1e-4, (t, k)
        orc.adam_deferred(W, M, V, Cn, sid, g_step, t, hp)
        np.testing.assert_array_equal(scene.counter[:n].cpu().numpy(), Cn)
        gw = scene.w[:, :n].cpu().numpy()
        gm = scene.m[:, :n].cpu().numpy()
        for k, s in GROUPS.items():
            if M[s].size:
                assert rel_group_error(gm, M, s) <= 2e-6, (t, k, rel_group_error(gm, M, s))
        err = np.abs(gw - W)
        assert np.all(err <= 2e-3 * 1e-3 + 1e-6 + 4e-7 * np.abs(W)), np.max(err)


def test_step_timing_spans(gs):
    """Stage timing inside gs_step: every span recorded, nested spans inside
    the step, and timing re-enabled between steps (a new event set) works."""
    c = scenes.cfg_small_step()
    P, cam = c["scene"], cam_f32(c["cams"][0])
    n = P.shape[1]
    scene = gs.GaussianScene(P, 0)
    ctx = make_ctx(gs, n, cam.width, cam.height, deg=0)
    tgt = torch.zeros(3, cam.height, cam.width, device="cuda")
    adam = gs.adam_struct()
    for rounds in range(2):
        ctx.timing_enable(4)
        for _ in range(3):
            ctx.step(scene, [cam], [tgt], adam)
        sp = ctx.timing_read(4)
        assert len(sp) == 3
        for x in sp:
            assert all(v >= 0 for v in x.values()), x
            assert x["cull"] + x["fwd"] + x["bwd"] + x["adam"] <= x["step"] * 1.01 + 1e-3
            assert x["adam_apply"] <= x["adam"] + 1e-3 and x["raster_bwd"] <= x["bwd"] + 1e-3
    ctx.timing_enable(0)
    ctx.step(scene, [cam], [tgt], adam)
    ctx.sync_status()
    assert scene.step == 7


def test_step_two_views_parity(gs, orc):
    """gs_step over two views (one fused rasterizer launch per direction): the
    loss is the sum of the views' L1 losses, the gradient of a Gaussian the sum
    of its views' gradients, and one optimizer step covers the union of the
    visible sets (§2.4 steps 1-6 with several views per iteration)."""
    P = scenes.uniform_cube_scene(6000, seed=41, sh_degree=1, log_scale_mean=-3.0)
    deg, tile = 1, (16, 16)
    n, D = P.shape[1], P.shape[0]
    cams = [cam_f32(scenes.camera_lookat((0.6, -0.2, -2.8), (0.3, 0.0, 0.0), 80, 60, 55.0, up=(0, -1, 0))),
            cam_f32(scenes.camera_lookat((-0.7, 0.3, -2.6), (-0.4, 0.1, 0.0), 72, 56, 60.0, up=(0, -1, 0)))]
    T = f32(scenes.uniform_cube_scene(n, seed=42, sh_degree=deg, log_scale_mean=-3.0))
    targets = [orc.render(T, deg, c, tile)["image"] for c in cams]
    scene = gs.GaussianScene(P, deg)
    ctx = make_ctx(gs, n, 80, 60, deg=deg, tile=tile, views=2)
    adam = gs.adam_struct(lr=1e-3, eps=1e-15)
    hp = hp32(orc, lr=1e-3, eps=1e-15)
    loss = ctx.step(scene, cams, [torch.as_tensor(t, dtype=torch.float32, device="cuda") for t in targets], adam)
    ctx.sync_status()
    W, M, V, Cn = f32(P), np.zeros((D, n)), np.zeros((D, n)), np.zeros(n, np.uint8)
    g = np.zeros((D, n))
    vis = np.zeros(n, bool)
    ref_loss = 0.0
    for c, t in zip(cams, targets):
        rr = orc.render_loss_backward(W, deg, c, t, tile)
        kept = rr["splats"]["keep"] == 1
        g[:, kept] += rr["grad"][:, kept]
        vis |= kept
        ref_loss += rr["loss"]
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    ids = np.nonzero(vis)[0].astype(np.int32)
    orc.adam_deferred(W, M, V, Cn, ids, g[:, ids], 1, hp)
    np.testing.assert_array_equal(scene.counter[:n].cpu().numpy(), Cn)
    gm = scene.m[:, :n].cpu().numpy().astype(np.float64)
    for k, sl in GROUPS.items():
        if M[sl].size:
            assert rel_group_error(gm, M, sl) <= 2e-4, (k, rel_group_error(gm, M, sl))


# ---------------------------------------------------------------------------- autograd

def test_autograd_function(gs, orc):
    P, cam, deg, tile = _case("cube_offaxis_sh3")
    camf = cam_f32(cam)
    ctx = make_ctx(gs, P.shape[1], camf.width, camf.height, deg=3)
    scene = gs.GaussianScene(P, deg, with_optimizer=False)
    ids, nv = ctx.cull(scene, camf)
    w = scene.w.detach().requires_grad_(True)
    scene.w = w
    img = gs.render(ctx, scene, camf, ids, nv)
    rng = np.random.default_rng(1)
    wimg = torch.as_tensor(rng.normal(size=img.shape), dtype=torch.float32, device="cuda")
    (g,) = torch.autograd.grad((img * wimg).sum(), w)
    r = orc.render(f32(P), deg, camf, tile)
    g_ref, _ = orc.backward(f32(P), deg, r["cam"], r["splats"], r["key_gid"], r["ranges"],
                            wimg.cpu().numpy().astype(np.float64))
    g_gpu = g[:, :P.shape[1]].cpu().numpy().astype(np.float64)
    errs = {k: rel_group_error(g_gpu, g_ref, s) for k, s in GROUPS.items()}
    assert max(errs.values()) <= 1e-4, errs


# ---------------------------------------------------------------------------- edge cases

def test_empty_view(gs):
    P = scenes.uniform_cube_scene(500, seed=0, sh_degree=0)
    cam = scenes.camera_from_pose(np.eye(3), (0.0, 0.0, -5.0), 32, 32, 60.0)   # cube behind the camera
    ctx = make_ctx(gs, 500, 32, 32, deg=0)
    scene = gs.GaussianScene(P, 0)
    ids, nv = ctx.cull(scene, cam)
    img = ctx.render_fwd(scene, cam, ids, nv)
    gc = ctx.render_bwd(torch.ones_like(img), 14)
    ctx.adam_deferred(scene, ids, nv, gc, gs.adam_struct())
    ctx.sync_status()
    assert nv.item() == 0
    assert img.abs().max().item() == 0.0
    assert int(scene.counter[:500].max().item()) == 1


def test_single_gaussian_and_ragged_n(gs, orc):
    for n in (1, 31, 33, 2049):
        P = scenes.uniform_cube_scene(n, seed=n, sh_degree=0, log_scale_mean=-2.0)
        cam = scenes.camera_from_pose(np.eye(3), (0.0, 0.0, 3.0), 40, 24, 60.0)
        camf = cam_f32(cam)
        ctx = make_ctx(gs, n, 40, 24, deg=0)
        scene = gs.GaussianScene(P, 0)
        ids, nv = ctx.cull(scene, camf)
        img = ctx.render_fwd(scene, camf, ids, nv)
        ctx.sync_status()
        r = orc.render(f32(P), 0, camf)
        kept = np.nonzero(r["splats"]["keep"])[0]
        np.testing.assert_array_equal(ids[:nv.item()].cpu().numpy(), kept)
        ex = _pixel_exclusions(r, ids[:nv.item()].cpu().numpy())
        err = np.abs(img.cpu().numpy() - r["image"])[:, ~ex]
        assert err.max() <= 1e-5


def test_capacity_overflow_is_reported(gs):
    from paper_2509_15645_b300 import _lib
    c = scenes.cfg_small_step()
    P, cam = c["scene"], c["cams"][0]
    ctx = make_ctx(gs, P.shape[1], 64, 64, deg=0, max_vis=100)
    scene = gs.GaussianScene(P, 0)
    ids, nv = ctx.cull(scene, cam)
    with pytest.raises(_lib.GsError) as e:
        ctx.sync_status()
    assert e.value.status == _lib.GS_ERR_CAPACITY
    assert nv.item() == 100
    ctx2 = make_ctx(gs, P.shape[1], 64, 64, deg=0, max_keys=1000)
    ids, nv = ctx2.cull(scene, cam)
    ctx2.render_fwd(scene, cam, ids, nv)
    with pytest.raises(_lib.GsError) as e:
        ctx2.sync_status()
    assert e.value.status == _lib.GS_ERR_CAPACITY
    ctx2.sync_status()   # cleared


def test_cull_timeout_is_reported_and_the_context_recovers(gs):
    """The cull blocks' bounded waits on their own TMA copies: with the first
    wait's limit at 0 every block gives up at once, lets its copies land and
    returns; GS_ERR_TIMEOUT is latched (gs_cull and a whole gs_step) with no
    fault, and with the default limit back the same context culls as before."""
    from paper_2509_15645_b300 import _lib
    c = scenes.cfg_small_step()
    P, cam = c["scene"], cam_f32(c["cams"][0])
    n = P.shape[1]
    ctx = make_ctx(gs, n, 64, 64, deg=0)
    scene = gs.GaussianScene(P, 0)
    ids_ref, nv_ref = ctx.cull(scene, cam)
    ctx.sync_status()
    ref = ids_ref[:int(nv_ref.item())].clone()
    adam = gs.adam_struct(lr=1e-3, eps=1e-15)
    tgt = torch.zeros(3, 64, 64, device="cuda")
    ctx.set_cull_wait_limit(0)
    ctx.cull(scene, cam)
    with pytest.raises(_lib.GsError) as e:
        ctx.sync_status()
    assert e.value.status == _lib.GS_ERR_TIMEOUT
    ctx.step(scene, [cam], [tgt], adam)
    with pytest.raises(_lib.GsError) as e:
        ctx.sync_status()
    assert e.value.status == _lib.GS_ERR_TIMEOUT
    ctx.set_cull_wait_limit(1 << 24)
    ids, nv = ctx.cull(scene, cam)
    ctx.sync_status()
    assert torch.equal(ids[:int(nv.item())], ref)


def test_raster_tma_timeout_is_reported(gs):
    """The TMA-staged rasterizer (variant 9) bounds its waits on its own bulk
    copies the same way: with the first wait's limit at 0 every warp gives up,
    lets its copies land and returns; GS_ERR_TIMEOUT is latched with no fault,
    and with the default limit back the render equals variant 7's bit for bit."""
    from paper_2509_15645_b300 import _lib
    P, cam, deg, _ = _case("tile8x4_ragged")
    camf = cam_f32(cam)
    n = P.shape[1]
    ctx = make_ctx(gs, n, camf.width, camf.height, deg=3, tile=(8, 4), list_records=1)
    scene = gs.GaussianScene(P, deg)
    ids, nv = ctx.cull(scene, camf)
    ctx.set_raster_variant(7)
    ref = ctx.render_fwd(scene, camf, ids, nv).clone()
    ctx.sync_status()
    ctx.set_raster_variant(9)
    ctx.set_cull_wait_limit(0)
    with pytest.raises(_lib.GsError) as e:
        ctx.render_fwd(scene, camf, ids, nv)       # the cull of the first line ran before the limit changed
        ctx.sync_status()
    assert e.value.status == _lib.GS_ERR_TIMEOUT
    ctx.set_cull_wait_limit(1 << 24)
    img = ctx.render_fwd(scene, camf, ids, nv)
    ctx.sync_status()
    assert torch.equal(img, ref)
