"""GPU parity of balance-aware image splitting (GS-Scale §4.4): the split
search against the oracle's, region renders stitched against the whole view,
and one training step over a view's two regions against the oracle's
whole-view step (the paper's claim: the split is mathematically equivalent).
This file sorts last so that a run stopping at its first failure has already
run every other test."""
import numpy as np
import pytest
import torch

from helpers import GROUPS, TIE_TOL, cam_f32, f32, hp32, pixel_exclusions, rel_group_error
from synth import scenes

pytestmark = pytest.mark.gpu

TILE = (8, 4)
DEG = 1


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2509_15645_b300 as gs
    return gs


def _scene(seed=51):
    """A cube of Gaussians with denser bands (x > 0.3, y < -0.2), so the
    balance point is off-centre; a 128x96 view sees 3837 of the 4000."""
    P = scenes.uniform_cube_scene(4000, seed=seed, sh_degree=DEG, log_scale_mean=-3.0)
    P[0] = np.where(P[0] < 0.3, P[0], P[0] * 0.2)
    P[1] = np.where(P[1] < -0.2, P[1] * 0.3, P[1])
    return P


def _cam():
    return cam_f32(scenes.camera_lookat((0.2, -0.1, -2.0), (0.0, 0.0, 0.0), 128, 96, 60.0, up=(0, -1, 0)))


def _ctx(gs, n, views=2, render_views=0):
    return gs.Context(max_gaussians=n, max_visible=n, max_keys=64 * n + 4096, max_width=128, max_height=96,
                      tile=TILE, max_views=views, max_sh_degree=DEG, render_views=render_views)


@pytest.mark.parametrize("axis", [0, 1])
def test_split_point_matches_oracle(gs, orc, axis):
    P = _scene()
    cam, n = _cam(), P.shape[1]
    ctx = _ctx(gs, n)
    scene = gs.GaussianScene(P, DEG)
    ax, split, counts = ctx.split_point(scene, cam, axis=axis, steps=5)
    ctx.sync_status()
    oc = orc.camera(cam, TILE)
    sp = orc.project(f32(P), DEG, oc)
    at, ref = orc.balance_split(sp, oc, axis, steps=5)
    assert ax == axis and split == at * TILE[axis], (split, at)
    ties = int(np.sum(sp["margin"] < TIE_TOL))
    assert abs(counts[0] - ref[0]) <= ties and abs(counts[1] - ref[1]) <= ties, (counts, ref, ties)


@pytest.mark.parametrize("axis,split", [(0, 56), (1, 48), (0, 8), (0, 61), (1, 37)])
def test_region_renders_stitch_to_the_view(gs, orc, axis, split):
    """Each region culls and renders on its own; placed side by side their
    images are the whole view's (oracle, FP64).  With the split on a tile
    boundary the union of their visible sets is the whole view's; elsewhere a
    region's last tile reaches past its pixels and may keep Gaussians that
    touch no pixel of it."""
    P = _scene()
    cam, n = _cam(), P.shape[1]
    ctx = _ctx(gs, n)
    scene = gs.GaussianScene(P, DEG)
    r = orc.render(f32(P), DEG, cam, TILE)
    img = np.zeros((3, cam.height, cam.width))
    vis = []
    for reg in gs.split_regions(cam, axis, split):
        ids, nv = ctx.cull(scene, reg)
        im = ctx.render_fwd(scene, reg, ids, nv)
        ctx.sync_status()
        img[:, reg.y0:reg.y0 + reg.height, reg.x0:reg.x0 + reg.width] = im.cpu().numpy()
        vis.append(ids[:int(nv.item())].cpu().numpy())
    union = np.union1d(vis[0], vis[1])
    ties = np.nonzero(r["splats"]["margin"] < TIE_TOL)[0]
    kept = np.nonzero(r["splats"]["keep"])[0]
    assert np.all(np.isin(np.setdiff1d(kept, union), ties))           # nothing the view keeps is lost
    if split % TILE[axis] == 0:
        assert np.all(np.isin(np.setxor1d(union, kept), ties))
    ex = pixel_exclusions(r, union)
    ok = ~ex[None, :, :].repeat(3, 0)
    assert ex.mean() < 0.03, ex.mean()
    err = np.abs(img - r["image"])
    assert err[ok].max() <= 1e-5, err[ok].max()


@pytest.mark.parametrize("render_views", [0, 1])
def test_split_step_matches_whole_view_step(gs, orc, render_views):
    """gs_step over a view's two regions (split where gs_split_point puts it,
    region targets cropped from the view's target) takes the whole view's
    step: loss = the view's L1 loss, one optimizer step over the union of the
    regions' visible sets with their summed gradients.  render_views = 1: the
    regions are rendered one after the other through one set of render
    buffers (the bounded working set of §4.4), with the same result."""
    P = _scene()
    cam, n, D = _cam(), P.shape[1], P.shape[0]
    T = f32(scenes.uniform_cube_scene(n, seed=60, sh_degree=DEG, log_scale_mean=-3.0))
    target = orc.render(T, DEG, cam, TILE)["image"]
    scene = gs.GaussianScene(P, DEG)
    ctx = _ctx(gs, n, render_views=render_views)
    adam = gs.adam_struct(lr=1e-3, eps=1e-15)
    hp = hp32(orc, lr=1e-3, eps=1e-15)
    regions = ctx.plan_split(scene, cam, adam, mem_limit=0.3)     # 3837 / 4000 visible: split
    assert regions is not None and len(regions) == 2
    assert ctx.plan_split(scene, cam, adam, mem_limit=0.99) is None
    tgt = torch.as_tensor(target, dtype=torch.float32, device="cuda")
    loss = ctx.step(scene, regions, [reg.crop(tgt) for reg in regions], adam)
    ctx.sync_status()
    assert scene.step == 1
    W, M, V, Cn = f32(P), np.zeros((D, n)), np.zeros((D, n)), np.zeros(n, np.uint8)
    rr = orc.render_loss_backward(W, DEG, cam, target, TILE)
    assert abs(loss.item() - rr["loss"]) <= 1e-5 * rr["loss"], (loss.item(), rr["loss"])
    # the regions' summed gradients the step used: the whole view's (per group,
    # Gaussians with a near-tie decision left out), then the oracle's step fed
    # those gradients, every entry within FP32 rounding
    good = ~(rr["splats"]["margin"] < TIE_TOL)          # Gaussians with no near-tie decision
    sid, sg = ctx.step_gradients(D)
    sid = sid.cpu().numpy().astype(np.int32)
    g_step = sg.cpu().numpy().astype(np.float64)
    kept = np.nonzero(rr["splats"]["keep"])[0]
    assert np.all(np.isin(np.setxor1d(sid, kept), np.nonzero(~good)[0]))
    g_full = np.zeros((D, n))
    g_full[:, sid] = g_step
    for k, sl in GROUPS.items():
        if M[sl].size:
            assert rel_group_error(g_full[:, good], rr["grad"][:, good], sl) <= 1e-4, k
    orc.adam_deferred(W, M, V, Cn, sid, g_step, 1, hp)
    np.testing.assert_array_equal(scene.counter[:n].cpu().numpy(), Cn)
    gm = scene.m[:, :n].cpu().numpy().astype(np.float64)
    for k, sl in GROUPS.items():
        if M[sl].size:
            assert rel_group_error(gm, M, sl) <= 2e-6, (k, rel_group_error(gm, M, sl))
    err = np.abs(scene.w[:, :n].cpu().numpy() - W)
    assert np.all(err <= 2e-3 * 1e-3 + 1e-6 + 4e-7 * np.abs(W)), np.max(err)


def test_region_and_split_argument_checks(gs):
    """Regions outside their full image, a split of a region, a context
    without two view slots and an unknown axis are refused before any launch."""
    from paper_2509_15645_b300 import _lib
    P = _scene()
    cam, n = _cam(), P.shape[1]
    ctx = _ctx(gs, n)
    scene = gs.GaussianScene(P, DEG)
    with pytest.raises(_lib.GsError):
        ctx.cull(scene, gs.RegionCamera(cam, 100, 0, 64, 96))          # x0 + width > 128
    with pytest.raises(_lib.GsError):
        ctx.split_point(scene, gs.RegionCamera(cam, 0, 0, 64, 96), axis=0)
    with pytest.raises(_lib.GsError):
        ctx.split_point(scene, cam, axis=2)
    with pytest.raises(_lib.GsError):
        _ctx(gs, n, views=1).split_point(scene, cam, axis=0)
