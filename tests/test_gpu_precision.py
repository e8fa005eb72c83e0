"""Error of the precision forms against the FP64 oracle, stated per result
(the image, each gradient group, each updated parameter group), for the plain
FP32 form and the BF16 form (SH coefficients and both moments stored as bf16,
geometry fp32, every computation fp32) with stochastic and with
round-to-nearest stores.

* One step from a shared state (the oracle is fed what the GPU stores): the
  image and the gradients are FP32 arithmetic on the same inputs in every form;
  the stored update carries the form's rounding.
* A training trajectory of 300 steps over changing views, the GPU forms and
  the FP64 oracle each following their own gradients from the same start:
  how far the parameters and the loss drift apart.

Run with -s to see the tables."""
import numpy as np
import pytest
import torch

from helpers import GROUPS, cam_f32, cancellation_bound, f32, hp32, pixel_exclusions, rel_group_error
from synth import scenes

pytestmark = pytest.mark.gpu

FORMS = ("fp32", "bf16_sr", "bf16_rn")


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2509_15645_b300 as gs
    return gs


def _prec(gs, form):
    return {"fp32": gs.GS_FP32, "bf16_sr": gs.GS_BF16_SH_MOM, "bf16_rn": gs.GS_BF16_SH_MOM_RN}[form]


def _state(scene, n):
    m, v = scene.moments()
    return (scene.params().cpu().numpy().astype(np.float64), m.cpu().numpy().astype(np.float64),
            v.cpu().numpy().astype(np.float64), scene.counter[:n].cpu().numpy().copy())


def _case(name):
    if name == "cube10k_64":
        P = scenes.uniform_cube_scene(10_000, seed=70, sh_degree=3, log_scale_mean=-3.0)
        cams = [scenes.camera_lookat(e, (0.0, 0.0, 0.0), 64, 64, 60.0, up=(0, -1, 0))
                for e in ((0.0, 0.0, -3.0), (0.8, -0.3, -2.8))]
        return P, [cam_f32(c) for c in cams], (16, 16)
    c = scenes.cfg_diff_check(n=200_000, width=512)
    cam = c["cams"][0]
    cam2 = scenes.camera_lookat((0.4, -0.2, -3.0), (0.0, 0.0, 0.0), 512, 512, 60.0, up=(0, -1, 0))
    return c["scene"], [cam_f32(cam), cam_f32(cam2)], (16, 16)


def _group_rel_max(a, b, rows):
    """max |a - b| / (|b| + 1e-3 max|b|) over a group of rows."""
    x, y = a[rows], b[rows]
    return float(np.max(np.abs(x - y) / (np.abs(y) + 1e-3 * np.abs(y).max() + 1e-30)))


@pytest.mark.parametrize("case", ["cube10k_64", "cube200k_512"])
def test_one_step_errors_per_result(gs, orc, case):
    P, cams, tile = _case(case)
    n, D, deg = P.shape[1], P.shape[0], 3
    T = f32(scenes.uniform_cube_scene(n, seed=71, sh_degree=deg, log_scale_mean=-3.0))
    targets = [orc.render(T, deg, c, tile)["image"] for c in cams]
    lr = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4]
    hp = hp32(orc, lr=lr, eps=1e-15)
    rows = []
    for form in FORMS:
        scene = gs.GaussianScene(P, deg, precision=_prec(gs, form))
        ctx = gs.Context(max_gaussians=n, max_visible=n, max_keys=64 * n + 4096, max_width=cams[0].width,
                         max_height=cams[0].height, tile=tile, max_sh_degree=deg)
        adam = gs.adam_struct(lr=lr, eps=1e-15, seed=4)
        tg = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in targets]
        for k in (0, 1, 0):                            # moments, and delays of 1 for part of the scene
            ctx.step(scene, [cams[k]], [tg[k]], adam)
        ctx.sync_status()
        t, cam = scene.step + 1, cams[1]
        W, M, V, Cn = _state(scene, n)
        Wcur, _, _ = orc.adam_materialize(W, M, V, Cn, t - 1, hp)
        rr = orc.render_loss_backward(Wcur, deg, cam, targets[1], tile)
        ids, nv = ctx.cull(scene, cam, adam)
        img = ctx.render_fwd(scene, cam, ids, nv, adam)
        ctx.sync_status()
        gids = ids[:int(nv.item())].cpu().numpy()
        ex = pixel_exclusions(rr, gids)
        ok = ~ex[None].repeat(3, 0)
        ierr_full = np.abs(img.cpu().numpy().astype(np.float64) - rr["image"])
        ierr = ierr_full[ok]
        # per pixel: 1e-5, plus what the cancellation in sigma allows for long splats
        bnd = 1e-5 + cancellation_bound(rr["splats"], cam.height, cam.width)[None].repeat(3, 0)
        over = float(np.max(ierr_full[ok] / bnd[ok]))
        dimg = rr["dimage"] * ok
        g_ref, _ = orc.backward(Wcur, deg, rr["cam"], rr["splats"], rr["key_gid"], rr["ranges"], dimg)
        gc = ctx.render_bwd(torch.as_tensor(dimg, dtype=torch.float32, device="cuda"), D)
        g_gpu = ctx.grad_scatter(scene, ids, nv, gc)[:, :n].cpu().numpy().astype(np.float64)
        # the step itself, against the oracle's from the same stored state; the
        # Gaussians whose gradient depends on a tie pixel are left out (counted)
        ctx.step(scene, [cam], [tg[1]], adam)
        ctx.sync_status()
        # the same step fed the gradients the GPU step used: the update's own error
        sid, sg = ctx.step_gradients(D)
        Ws, Ms, Vs, Cs = W.copy(), M.copy(), V.copy(), Cn.copy()
        orc.adam_deferred(Ws, Ms, Vs, Cs, sid.cpu().numpy().astype(np.int32), sg.cpu().numpy().astype(np.float64),
                          t, hp)
        orc.adam_deferred(W, M, V, Cn, gids.astype(np.int32), rr["grad"][:, gids], t, hp)
        gw, gm, gv, _ = _state(scene, n)
        upd = {k: float(np.abs(gw[s] - Ws[s]).max() / hp.lr[list(GROUPS).index(k)]) for k, s in GROUPS.items()}
        keep = ~np.any(g_ref != rr["grad"], axis=0)
        W, M, V, gw, gm, gv = (x[:, keep] for x in (W, M, V, gw, gm, gv))
        row = {"case": case, "form": form, "image_max": float(ierr.max()), "image_mean": float(ierr.mean()),
               "image_p9999": float(np.quantile(ierr, 0.9999)), "image_over_bound": over,
               "image_frac_gt_1e-5": float(np.mean(ierr > 1e-5)), "tie_pixels": float(ex.mean()),
               "tie_affected_gaussians": int((~keep).sum())}
        for k, s in GROUPS.items():
            row[f"upd_{k}"] = upd[k]
            row[f"grad_{k}"] = rel_group_error(g_gpu, g_ref, s)
            row[f"w_{k}_max"] = float(np.abs(gw[s] - W[s]).max())
            row[f"w_{k}_rel_lr"] = float(np.abs(gw[s] - W[s]).max() / hp.lr[list(GROUPS).index(k)])
            row[f"m_{k}"] = _group_rel_max(gm, M, s)
            row[f"v_{k}"] = _group_rel_max(gv, V, s)
        rows.append(row)
    print(f"\n{case}: one step from a shared state, error against the FP64 oracle")
    print(f"{'form':8s} {'img max':>9s} {'img mean':>9s} {'p99.99':>9s} {'>1e-5':>8s}  " +
          " ".join(f"{'g_' + k:>10s}" for k in GROUPS))
    for r in rows:
        print(f"{r['form']:8s} {r['image_max']:9.2e} {r['image_mean']:9.2e} {r['image_p9999']:9.2e} "
              f"{r['image_frac_gt_1e-5']:8.1e}  " + " ".join(f"{r['grad_' + k]:10.2e}" for k in GROUPS))
    print(f"{'form':8s} |w - w_ref| / lr per group, then max rel. error of m and v (SH rest)")
    for r in rows:
        print(f"{r['form']:8s} " + " ".join(f"{r['w_' + k + '_rel_lr']:9.2e}" for k in GROUPS) +
              f"   m {r['m_sh_rest']:.2e} v {r['v_sh_rest']:.2e}   ({r['tie_affected_gaussians']} tie-affected left out)")
    print(f"{'form':8s} |w - w_ref| / lr per group, the oracle's step fed the GPU step's own gradients (the update alone)")
    for r in rows:
        print(f"{r['form']:8s} " + " ".join(f"{r['upd_' + k]:9.2e}" for k in GROUPS))
    for row in rows:
        # the forms' stated bounds: FP32 image (1e-5, plus the cancellation bound
        # of long splats) and FP32 gradients, in every form; the update from the
        # same gradients: FP32 rounding in fp32 (geometry in every form), one
        # bf16 ulp of the stored SH values (a few lr at these rates) otherwise
        assert row["image_over_bound"] <= 1.0, row
        geo_lim = 2e-3
        assert max(row[f"upd_{k}"] for k in ("mean", "log_scale", "quat", "opacity")) <= geo_lim, row
        if row["form"] == "fp32":
            assert max(row[f"upd_{k}"] for k in ("sh_dc", "sh_rest")) <= geo_lim, row
        assert max(row[f"grad_{k}"] for k in GROUPS) <= 1e-4, row
        lim = 2e-4 if row["form"] == "fp32" else 2.0 ** -7 * 1.01
        for k in ("sh_dc", "sh_rest"):
            assert row[f"m_{k}"] <= lim + 2e-4 and row[f"v_{k}"] <= lim + 4e-4, (row["form"], k, row)


def test_trajectory_error_statistics(gs, orc):
    """300 deferred-Adam steps over 8 changing views of a 50k-Gaussian
    heightfield (SH degree 3, 128x96), each form following its own gradients,
    against the FP64 oracle's own trajectory from the same start: relative
    parameter drift per group (RMS of w - w_oracle over RMS of w_oracle - w0)
    and loss drift at steps 10, 100 and 300."""
    n, deg, tile = 50_000, 3, (8, 8)
    P = scenes.heightfield_scene(n, seed=80, half_extent=30.0, amplitude=3.0, wavelength=(12.0, 15.0),
                                 n_clusters=2, cluster_size=5000, sh_degree=deg)
    Tg = f32(scenes.heightfield_scene(n, seed=81, half_extent=30.0, amplitude=3.0, wavelength=(12.0, 15.0),
                                      n_clusters=2, cluster_size=5000, sh_degree=deg))
    cams = [cam_f32(scenes.camera_aerial((12 * np.cos(a), 12 * np.sin(a), 30.0), a, -np.pi / 2 + 0.3, 128, 96, 60.0))
            for a in np.linspace(0, 2 * np.pi, 9)[:8]]
    targets = [orc.render(Tg, deg, c, tile)["image"] for c in cams]
    lr = [1.6e-4 * 10, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4]
    hp = hp32(orc, lr=lr, eps=1e-15)
    steps, checks = 300, (10, 100, 300)
    # the FP64 oracle's trajectory (deferred Adam with its tables, its own renders and gradients)
    W, M, V, Cn = f32(P), np.zeros_like(f32(P)), np.zeros_like(f32(P)), np.zeros(n, np.uint8)
    ref, ref_loss = {}, {}
    for t in range(1, steps + 1):
        k = (t - 1) % len(cams)
        Wc, _, _ = orc.adam_materialize(W, M, V, Cn, t - 1, hp)
        rr = orc.render_loss_backward(Wc, deg, cams[k], targets[k], tile)
        ref_loss[t] = rr["loss"]
        kept = np.nonzero(rr["splats"]["keep"])[0].astype(np.int32)
        orc.adam_deferred(W, M, V, Cn, kept, rr["grad"][:, kept], t, hp)
        if t in checks:
            ref[t] = orc.adam_materialize(W, M, V, Cn, t, hp)[0]
    W0 = f32(P)
    table = []
    for form in FORMS:
        scene = gs.GaussianScene(P, deg, precision=_prec(gs, form))
        ctx = gs.Context(max_gaussians=n, max_visible=n, max_keys=64 * n, max_width=128, max_height=96, tile=tile,
                         max_sh_degree=deg)
        adam = gs.adam_struct(lr=lr, eps=1e-15, seed=6)
        tg = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in targets]
        loss = torch.zeros(1, device="cuda")
        for t in range(1, steps + 1):
            k = (t - 1) % len(cams)
            ctx.step(scene, [cams[k]], [tg[k]], adam, loss=loss)
            if t in checks:
                lv = loss.item()
                wo, _, _ = ctx.materialize(scene, adam)
                wg = wo[:, :n].cpu().numpy().astype(np.float64)
                row = {"form": form, "step": t, "loss_rel": abs(lv - ref_loss[t]) / ref_loss[t]}
                for g, s in GROUPS.items():
                    moved = np.sqrt(np.mean((ref[t][s] - W0[s]) ** 2)) + 1e-30
                    row[g] = float(np.sqrt(np.mean((wg[s] - ref[t][s]) ** 2)) / moved)
                table.append(row)
        ctx.sync_status()
    print("\ntrajectory drift against the FP64 oracle: RMS(w - w_oracle) / RMS(w_oracle - w0) per group, "
          "and |loss - loss_oracle| / loss_oracle")
    print(f"{'form':8s} {'step':>5s} {'loss':>9s} " + " ".join(f"{g:>9s}" for g in GROUPS))
    for r in table:
        print(f"{r['form']:8s} {r['step']:5d} {r['loss_rel']:9.2e} " + " ".join(f"{r[g]:9.2e}" for g in GROUPS))
    for r in table:
        assert r["loss_rel"] < 0.05, r                 # every form trains the same way
    fp = {r["step"]: r for r in table if r["form"] == "fp32"}
    assert all(fp[t]["loss_rel"] < 1e-2 for t in checks), fp
