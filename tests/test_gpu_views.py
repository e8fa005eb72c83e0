"""GPU parity of the deferred restore over changing views (§4.3.3 parameter
forwarding with the Eq. 3 catch-up, §4.2.1 selective offloading).

A training run cycles through views of one heightfield that overlap only in
part, so each view sees Gaussians deferred for 0 to several steps, and (with
a small counter bound) Gaussians that no view sees are caught up through the
counter bound.  At every step the oracle is fed the GPU's stored state (one-
step parity, since atomics make FP32 gradients run-dependent):

* resident scenes: the GPU's cull, render and backward with the restore (the
  gather restores each visible Gaussian on the fly) against the oracle's
  render of the materialised parameters -- cull set, image, gradients -- then
  the whole gs_step against the oracle's deferred Adam step;
* host-tier scenes (SH rows streamed through the staging ring): the loss of
  gs_step against the oracle's, and the stored state after the step.
"""
import numpy as np
import pytest
import torch

from helpers import GROUPS, TIE_TOL, cam_f32, f32, hp32, pixel_exclusions, rel_group_error
from synth import scenes

pytestmark = pytest.mark.gpu

N, DEG, TILE = 12_000, 3, (8, 8)
LR = [1e-3, 2e-3, 2e-3, 1e-2, 5e-3, 1e-3]
# the view of each step: overlapping views in an irregular order, so delays of 1 to 5 steps occur
ORDER = [0, 1, 2, 3, 0, 2, 1, 3, 3, 0, 1, 2]


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2509_15645_b300 as gs
    return gs


def _views():
    return [cam_f32(scenes.camera_aerial((9 * np.cos(a), 9 * np.sin(a), 35.0), a, -np.pi / 2 + 0.35, 96, 72, 55.0))
            for a in np.linspace(0, 2 * np.pi, 5)[:4]]


def _scene(seed):
    return scenes.heightfield_scene(N, seed=seed, half_extent=50.0, amplitude=5.0, wavelength=(20.0, 25.0),
                                    n_clusters=2, cluster_size=2000, sh_degree=DEG)


def _targets(orc, cams):
    T = f32(_scene(42))
    return [orc.render(T, DEG, c, TILE)["image"] for c in cams]


def _state(scene, n):
    """The stored (w, m, v, counter) as float64 / uint8 arrays [D][n]."""
    m, v = scene.moments()
    return (scene.params().cpu().numpy().astype(np.float64), m.cpu().numpy().astype(np.float64),
            v.cpu().numpy().astype(np.float64), scene.counter[:n].cpu().numpy().copy())


def _tie_affected(orc, Wcur, rr, ex):
    """Gaussians whose oracle gradient changes when the tie pixels are weighted
    0: a decision there may go the other way in FP32, so their step is not
    determined to FP32 accuracy (excluded from the state comparison, counted)."""
    g_m, _ = orc.backward(Wcur, DEG, rr["cam"], rr["splats"], rr["key_gid"], rr["ranges"], rr["dimage"] * ~ex[None])
    return np.any(g_m != rr["grad"], axis=0), g_m


def _check_step(orc, ctx, scene, n, t, prec_bf16, W, M, V, Cn, gids, grad, hp, lr, opt=None, skip=None):
    """The GPU's state after step t against the oracle's deferred step from the
    stored state (W, M, V, Cn), fed the gradients the GPU step used
    (gs_step_gradients), so the comparison is of the update alone: FP32
    rounding of each term, or in the bf16 forms one bf16 ulp (stochastic
    rounding picks either neighbour) plus the step's share.  Separately, those
    gradients against the oracle's (`grad`, for the visible set `gids`) per
    group within 1e-4, leaving out `skip` (tie-affected Gaussians, whose FP32
    gradient may follow a decision the other way).  opt: None (Adam),
    ("adamw", weight decay) or ("sgdm", momentum)."""
    D = W.shape[0]
    sid, sg = ctx.step_gradients(D)
    sid = sid.cpu().numpy().astype(np.int32)
    g_step = sg.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(sid, np.sort(gids))          # the step saw the cull's visible set
    g_gpu = np.zeros((D, n))
    g_gpu[:, sid] = g_step
    keep = np.ones(n, bool) if skip is None else ~skip
    for k, s in GROUPS.items():
        e = rel_group_error(g_gpu[:, keep], grad[:, keep], s)
        assert e <= 1e-4, (t, k, e)
    W0 = W.copy()
    if opt is None:
        orc.adam_deferred(W, M, V, Cn, sid, g_step, t, hp)
    elif opt[0] == "adamw":
        orc.adamw_deferred(W, M, V, Cn, sid, g_step, t, hp, opt[1])
    else:
        orc.sgdm_deferred(W, M, Cn, sid, g_step, hp.lr, opt[1], max_defer=hp.max_defer)
    gw, gm, gv, gc = _state(scene, n)
    np.testing.assert_array_equal(gc, Cn)
    lr_row = np.array([lr[0]] * 3 + [lr[1]] * 3 + [lr[2]] * 4 + [lr[3]] + [lr[4]] * 3 + [lr[5]] * (D - 14))[:, None]
    if not prec_bf16:
        for k, s in GROUPS.items():
            assert rel_group_error(gm, M, s) <= 2e-6, (t, k, rel_group_error(gm, M, s))
        if opt is not None and opt[0] == "sgdm":
            np.testing.assert_array_equal(gv, V)      # momentum SGD keeps no v
        err = np.abs(gw - W)
        bound = 2e-3 * lr_row + 1e-6 + 4e-7 * np.abs(W)
        assert np.all(err <= bound), (t, np.max(err / bound), np.unravel_index(np.argmax(err / bound), err.shape))
    else:
        ub = 2.0 ** -7
        for k, s in GROUPS.items():
            sm, sv = np.abs(M[s]).max() + 1e-30, np.abs(V[s]).max() + 1e-30
            assert np.all(np.abs(gm[s] - M[s]) <= ub * np.abs(M[s]) + 2e-4 * sm), (t, k, "m")
            assert np.all(np.abs(gv[s] - V[s]) <= ub * np.abs(V[s]) + 4e-4 * sv), (t, k, "v")
        err = np.abs(gw - W)
        geo = np.arange(D)[:, None] < 11
        bound = np.where(geo, 2e-3 * lr_row + 1e-6 + 4e-7 * np.abs(W),
                         ub * np.abs(W) + 2 * ub * lr_row * (t + 1) + 1e-7)
        assert np.all(err <= bound), (t, np.max(err / bound))
    return np.mean(np.abs(W - W0) > 0)


@pytest.mark.parametrize("bf16,opt", [(False, "adam"), (True, "adam"), (False, "adamw"), (False, "sgdm")])
def test_restore_over_changing_views(gs, orc, bf16, opt):
    """Resident scene, fp32 or the bf16 form (counter bound 15); Adam, and the
    deferred AdamW and momentum SGD of §4.3 in fp32."""
    from paper_2509_15645_b300 import _lib
    cams = _views()
    targets = _targets(orc, cams)
    P = _scene(41)
    prec = gs.GS_BF16_SH_MOM if bf16 else gs.GS_FP32
    scene = gs.GaussianScene(P, DEG, precision=prec)
    ctx = gs.Context(max_gaussians=N, max_visible=N, max_keys=64 * N, max_width=96, max_height=72, tile=TILE,
                     max_sh_degree=DEG)
    wd, mu = 0.05, 0.9
    kind = {"adam": _lib.GS_OPT_ADAM, "adamw": _lib.GS_OPT_ADAMW, "sgdm": _lib.GS_OPT_SGDM}[opt]
    adam = gs.adam_struct(lr=LR, eps=1e-15, seed=9, optimizer=kind, weight_decay=wd, beta1=mu if opt == "sgdm" else 0.9)
    hp = hp32(orc, lr=LR, eps=1e-15)
    ospec = None if opt == "adam" else ((opt, float(np.float32(wd))) if opt == "adamw" else (opt, float(np.float32(mu))))
    tg = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in targets]
    delays = []
    for t, k in enumerate(ORDER, start=1):
        cam = cams[k]
        W, M, V, Cn = _state(scene, N)
        if opt == "adamw":
            Wcur, _, _ = orc.adamw_materialize(W, M, V, Cn, t - 1, hp, ospec[1])
        elif opt == "sgdm":
            Wcur, _ = orc.sgdm_materialize(W, M, Cn, hp.lr, ospec[1], max_defer=hp.max_defer)
        else:
            Wcur, _, _ = orc.adam_materialize(W, M, V, Cn, t - 1, hp)
        rr = orc.render_loss_backward(Wcur, DEG, cam, targets[k], TILE)
        # cull + render + backward with the restore of the coming step
        ids, nv = ctx.cull(scene, cam, adam)
        img = ctx.render_fwd(scene, cam, ids, nv, adam)
        ctx.sync_status()
        gids = ids[:int(nv.item())].cpu().numpy()
        sp = rr["splats"]
        diff = np.setxor1d(gids, np.nonzero(sp["keep"])[0])
        assert np.all(sp["margin"][diff] < TIE_TOL), (t, diff[sp["margin"][diff] >= TIE_TOL][:8])
        ex = pixel_exclusions(rr, gids)
        assert ex.mean() < 0.03
        ok = ~ex[None].repeat(3, 0)
        ierr = np.abs(img.cpu().numpy().astype(np.float64) - rr["image"])
        assert ierr[ok].max() <= 1e-5, (t, ierr[ok].max())
        # gradients with the tie pixels weighted 0 on both sides (a decision at
        # FP32 resolution there may go either way and move whole gradients)
        dimg = rr["dimage"] * ok
        affected, g_ref = _tie_affected(orc, Wcur, rr, ex)
        gc = ctx.render_bwd(torch.as_tensor(dimg, dtype=torch.float32, device="cuda"), scene.D)
        full = ctx.grad_scatter(scene, ids, nv, gc)
        ctx.sync_status()
        g_gpu = full[:, :N].cpu().numpy().astype(np.float64)
        errs = {g: rel_group_error(g_gpu, g_ref, s) for g, s in GROUPS.items()}
        assert max(errs.values()) <= 1e-4, (t, errs, int(ex.sum()))
        d = Cn[gids]
        delays.append(d)
        if t > 1 and ORDER[t - 2] != k:
            assert np.mean(d > 0) > 0.1, (t, np.mean(d > 0))
        # the whole step (graph) from the same state
        loss = ctx.step(scene, [cam], [tg[k]], adam)
        ctx.sync_status()
        assert abs(loss.item() - rr["loss"]) <= 1e-5 * rr["loss"] + 1e-7, (t, loss.item(), rr["loss"])
        moved = _check_step(orc, ctx, scene, N, t, bf16, W, M, V, Cn, gids.astype(np.int32), rr["grad"], hp, LR, ospec,
                            skip=affected)
        assert affected.mean() < 0.02, (t, affected.mean())
        assert moved > 0.02
    d = np.concatenate(delays)
    hist = np.bincount(d, minlength=16)
    assert np.count_nonzero(hist[1:]) >= 3, hist          # several different delays were restored
    print(f"delays of the visible Gaussians over {len(ORDER)} steps: {hist[:8].tolist()}")


@pytest.mark.parametrize("prec_name", ["GS_FP32", "GS_BF16_SH_MOM"])
def test_host_tier_over_changing_views(gs, orc, prec_name):
    """Host-tier scene (SH rows streamed through a ring smaller than the
    scene) with a counter bound of 5, so never-visible Gaussians are stepped
    through the bound: loss and stored state after each gs_step against the
    oracle from the same stored state."""
    cams = _views()
    targets = _targets(orc, cams)
    P = _scene(41)
    prec = getattr(gs, prec_name)
    bf16 = prec != gs.GS_FP32
    scene = gs.GaussianScene(P, DEG, precision=prec, tier=gs.GS_TIER_HOST_SH)
    ctx = gs.Context(max_gaussians=N, max_visible=N, max_keys=64 * N, max_width=96, max_height=72, tile=TILE,
                     max_sh_degree=DEG, stage_chunks=10, chunk_shift=10, stage_elem_bytes=2 if bf16 else 4)
    adam = gs.adam_struct(lr=LR, eps=1e-15, seed=9, max_defer=5)
    hp = hp32(orc, lr=LR, eps=1e-15, max_defer=5)
    tg = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in targets]
    saw_bound = False
    for t, k in enumerate(ORDER, start=1):
        W, M, V, Cn = _state(scene, N)
        Wcur, _, _ = orc.adam_materialize(W, M, V, Cn, t - 1, hp)
        rr = orc.render_loss_backward(Wcur, DEG, cams[k], targets[k], TILE)
        ids, nv = ctx.cull(scene, cams[k], adam)
        ctx.sync_status()
        gids = ids[:int(nv.item())].cpu().numpy().astype(np.int32)
        sp = rr["splats"]
        diff = np.setxor1d(gids, np.nonzero(sp["keep"])[0])
        assert np.all(sp["margin"][diff] < TIE_TOL), t
        if t > 1 and ORDER[t - 2] != k:
            assert np.mean(Cn[gids] > 0) > 0.1
        saw_bound |= bool(np.any(Cn == 5))
        loss = ctx.step(scene, [cams[k]], [tg[k]], adam)
        ctx.sync_status()          # waits for the write-backs too
        assert abs(loss.item() - rr["loss"]) <= 1e-5 * rr["loss"] + 1e-7, (t, loss.item(), rr["loss"])
        affected, _ = _tie_affected(orc, Wcur, rr, pixel_exclusions(rr, gids))
        assert affected.mean() < 0.02, (t, affected.mean())
        _check_step(orc, ctx, scene, N, t, bf16, W, M, V, Cn, gids, rr["grad"], hp, LR, skip=affected)
        staged, _ = ctx.host_tier_stats()
        assert 0 < staged <= (N + 1023) // 1024
    assert saw_bound


def _cpu_tier(gs, P, max_defer, opt="adam"):
    from paper_2509_15645_b300 import _lib
    scene = gs.GaussianScene(P, DEG, tier=gs.GS_TIER_HOST_CPU_OPT)
    ctx = gs.Context(max_gaussians=N, max_visible=N, max_keys=64 * N, max_width=96, max_height=72, tile=TILE,
                     max_sh_degree=DEG, cpu_opt=1)
    kind = {"adam": _lib.GS_OPT_ADAM, "adamw": _lib.GS_OPT_ADAMW, "sgdm": _lib.GS_OPT_SGDM}[opt]
    adam = gs.adam_struct(lr=LR, eps=1e-15, seed=9, max_defer=max_defer, optimizer=kind, weight_decay=0.05,
                          beta1=0.9)
    return scene, ctx, adam


@pytest.mark.parametrize("opt", ["adam", "adamw", "sgdm"])
def test_cpu_optimizer_tier_over_changing_views(gs, orc, opt):
    """The paper's offloaded configuration (GS_TIER_HOST_CPU_OPT: SH planes
    stepped on the host cores, geometry on the device), synchronised after
    every step so nothing is held: loss and stored state after each gs_step
    against the oracle from the same stored state (counter bound 5)."""
    cams = _views()
    targets = _targets(orc, cams)
    scene, ctx, adam = _cpu_tier(gs, _scene(41), 5, opt)
    hp = hp32(orc, lr=LR, eps=1e-15, max_defer=5)
    ospec = None if opt == "adam" else (opt, float(np.float32(0.05 if opt == "adamw" else 0.9)))
    tg = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in targets]
    for t, k in enumerate(ORDER, start=1):
        W, M, V, Cn = _state(scene, N)
        if opt == "adamw":
            Wcur, _, _ = orc.adamw_materialize(W, M, V, Cn, t - 1, hp, ospec[1])
        elif opt == "sgdm":
            Wcur, _ = orc.sgdm_materialize(W, M, Cn, hp.lr, ospec[1], max_defer=hp.max_defer)
        else:
            Wcur, _, _ = orc.adam_materialize(W, M, V, Cn, t - 1, hp)
        rr = orc.render_loss_backward(Wcur, DEG, cams[k], targets[k], TILE)
        ids, nv = ctx.cull(scene, cams[k], adam)
        ctx.sync_status()
        gids = ids[:int(nv.item())].cpu().numpy().astype(np.int32)
        if t > 1 and ORDER[t - 2] != k:
            assert np.mean(Cn[gids] > 0) > 0.1
        loss = ctx.step(scene, [cams[k]], [tg[k]], adam)
        ctx.sync_status()          # applies the step's SH update on the host
        assert abs(loss.item() - rr["loss"]) <= 1e-5 * rr["loss"] + 1e-7, (t, loss.item(), rr["loss"])
        affected, _ = _tie_affected(orc, Wcur, rr, pixel_exclusions(rr, gids))
        assert affected.mean() < 0.02, (t, affected.mean())
        _check_step(orc, ctx, scene, N, t, False, W, M, V, Cn, gids, rr["grad"], hp, LR, ospec, skip=affected)
        st = ctx.cpu_tier_stats()
        assert st["rows"] == len(gids) and st["held_members"] >= len(gids)


def test_cpu_optimizer_tier_pipelined_trajectory(gs, orc):
    """The same configuration run as the paper pipelines it: no synchronisation
    between steps, so every step forwards its visible Gaussians from the host
    planes plus the previous step's held update while a worker applies that
    update.  Each step's loss against an FP64 oracle trajectory run alongside
    (its own gradients), and the state at the end (after gs_sync_status
    applies the last held update) against the oracle's state."""
    cams = _views()
    targets = _targets(orc, cams)
    P = _scene(41)
    scene, ctx, adam = _cpu_tier(gs, P, 5)
    hp = hp32(orc, lr=LR, eps=1e-15, max_defer=5)
    tg = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in targets]
    W0 = f32(P)
    W, M, V = W0.copy(), np.zeros_like(W0), np.zeros_like(W0)
    C = np.zeros(N, np.uint8)
    losses = []
    for t, k in enumerate(ORDER, start=1):
        Wcur, _, _ = orc.adam_materialize(W, M, V, C, t - 1, hp)
        rr = orc.render_loss_backward(Wcur, DEG, cams[k], targets[k], TILE)
        gids = np.nonzero(rr["splats"]["keep"])[0].astype(np.int32)
        orc.adam_deferred(W, M, V, C, gids, rr["grad"][:, gids], t, hp)
        losses.append((ctx.step(scene, [cams[k]], [tg[k]], adam), rr["loss"]))
    ctx.sync_status()
    for t, (lg, lo) in enumerate(losses, start=1):
        assert abs(lg.item() - lo) <= 2e-5 * lo + 1e-7, (t, lg.item(), lo)
    gw, gm, gv, gc = _state(scene, N)
    np.testing.assert_array_equal(gc, C)
    for g, s in GROUPS.items():
        moved = np.sqrt(np.mean((W[s] - W0[s]) ** 2))
        drift = np.sqrt(np.mean((gw[s] - W[s]) ** 2))
        assert drift <= 3e-2 * moved + 1e-9, (g, drift, moved)


def test_cpu_optimizer_tier_two_views_per_step(gs, orc):
    """The host-core optimizer configuration with two views per step (the
    visible ids are the union of the views', the forwarded rows and the
    gradients follow the union's order): the loss (sum of the views' L1
    losses), the union's summed gradients and the stored state after each step
    against the oracle from the same stored state (counter bound 5)."""
    cams = _views()
    targets = _targets(orc, cams)
    P = _scene(41)
    scene = gs.GaussianScene(P, DEG, tier=gs.GS_TIER_HOST_CPU_OPT)
    ctx = gs.Context(max_gaussians=N, max_visible=N, max_keys=64 * N, max_width=96, max_height=72, tile=TILE,
                     max_sh_degree=DEG, max_views=2, cpu_opt=1)
    adam = gs.adam_struct(lr=LR, eps=1e-15, seed=9, max_defer=5)
    hp = hp32(orc, lr=LR, eps=1e-15, max_defer=5)
    tg = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in targets]
    for t, pair in enumerate([(0, 1), (2, 3), (1, 2), (3, 0), (0, 2), (1, 3)], start=1):
        W, M, V, Cn = _state(scene, N)
        Wcur, _, _ = orc.adam_materialize(W, M, V, Cn, t - 1, hp)
        grad = np.zeros((W.shape[0], N))
        affected = np.zeros(N, bool)
        gids, ref_loss = [], 0.0
        for k in pair:
            rr = orc.render_loss_backward(Wcur, DEG, cams[k], targets[k], TILE)
            ids, nv = ctx.cull(scene, cams[k], adam)
            ctx.sync_status()
            g = ids[:int(nv.item())].cpu().numpy().astype(np.int32)
            gids.append(g)
            grad[:, g] += rr["grad"][:, g]
            affected |= _tie_affected(orc, Wcur, rr, pixel_exclusions(rr, g))[0]
            ref_loss += rr["loss"]
        union = np.union1d(gids[0], gids[1]).astype(np.int32)
        loss = ctx.step(scene, [cams[k] for k in pair], [tg[k] for k in pair], adam)
        ctx.sync_status()
        assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss + 1e-7, (t, loss.item(), ref_loss)
        assert affected.mean() < 0.04, (t, affected.mean())
        _check_step(orc, ctx, scene, N, t, False, W, M, V, Cn, union, grad, hp, LR, skip=affected)
        st = ctx.cpu_tier_stats()
        assert st["rows"] == len(union)
