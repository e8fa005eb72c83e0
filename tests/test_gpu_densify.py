"""GPU densification on deferred state (gs_densify, §2.4 step 7 with §4.3)
against the oracle's densify from the same stored state: the same clones,
splits and prunes (bit-exact counts and order, counters bit-exact), and the
new scene's parameters and moments within FP32 rounding of the FP64 values
(bf16 stores within one bf16 ulp)."""
import numpy as np
import pytest
import torch

from helpers import cam_f32, hp32
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2509_15645_b300 as gs
    return gs


def _trained_scene(gs, orc, prec, n=20_000, deg=1, steps=5):
    """A scene after a few deferred steps over two views (delays 0..4)."""
    P = scenes.uniform_cube_scene(n, seed=90, sh_degree=deg, log_scale_mean=-3.0, log_scale_std=0.8)
    P[10] = np.random.default_rng(91).normal(-1.0, 2.5, n)          # a spread of opacities: some get pruned
    # two narrow views of different parts of the cube: ~20% of the Gaussians
    # neither sees, ~40% only one, so counters run up between the two
    cams = [cam_f32(scenes.camera_lookat(e, la, 64, 48, 25.0, up=(0, -1, 0)))
            for e, la in (((0.0, 0.0, -3.0), (-0.5, 0.0, 0.0)), ((1.6, -0.4, -2.5), (0.5, 0.1, 0.0)))]
    T = np.asarray(scenes.uniform_cube_scene(n, seed=92, sh_degree=deg), np.float64)
    tg = [torch.as_tensor(orc.render(T, deg, c, (16, 16))["image"], dtype=torch.float32, device="cuda") for c in cams]
    scene = gs.GaussianScene(P, deg, precision=prec)
    ctx = gs.Context(max_gaussians=n, max_visible=n, max_keys=64 * n, max_width=64, max_height=48, tile=(16, 16),
                     max_sh_degree=deg)
    adam = gs.adam_struct(lr=[2e-3, 5e-3, 1e-3, 5e-2, 2.5e-3, 1e-3], eps=1e-15, seed=3)
    for t in range(steps):
        ctx.step(scene, [cams[t % 2]], [tg[t % 2]], adam)
    ctx.sync_status()
    return ctx, scene, adam


@pytest.mark.parametrize("prec_name", ["GS_FP32", "GS_BF16_SH_MOM"])
def test_densify_matches_oracle(gs, orc, prec_name):
    prec = getattr(gs, prec_name)
    bf16 = prec != gs.GS_FP32
    ctx, scene, adam = _trained_scene(gs, orc, prec)
    n, D = scene.n, scene.D
    hp = hp32(orc, lr=[2e-3, 5e-3, 1e-3, 5e-2, 2.5e-3, 1e-3], eps=1e-15)
    m, v = scene.moments()
    W = scene.params().cpu().numpy().astype(np.float64)
    M, V = m.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    Cn = scene.counter[:n].cpu().numpy().copy()
    assert np.count_nonzero(Cn) > n // 10                            # deferred rows take part
    rng = np.random.default_rng(93)
    denom = rng.integers(0, 6, n).astype(np.float32)
    accum = (denom * np.abs(rng.normal(0.0, 3e-4, n))).astype(np.float32)
    normals = rng.standard_normal((2, 3, n)).astype(np.float32)
    # thresholds away from every decision's tie (FP32 against FP64)
    wc, _, _ = orc.adam_materialize(W, M, V, Cn, scene.step, hp)
    g = np.where(denom > 0, accum.astype(np.float64) / np.maximum(denom, 1), 0.0)
    smax = np.exp(wc[3:6]).max(axis=0)
    thr, pd, min_op = 2e-4, 0.01, 0.005
    # the split threshold pd * extent in the widest gap between the sorted
    # largest scales near the median of the densified Gaussians' (no tie)
    allv = np.sort(smax)
    i = int(np.searchsorted(allv, np.median(smax[g >= thr])))
    win = allv[max(i - 20, 0):i + 21]
    j = int(np.argmax(np.diff(win)))
    extent = float(np.sqrt(win[j] * win[j + 1]) / pd)
    opac = 1.0 / (1.0 + np.exp(-wc[10]))
    for q, lim in ((g, thr), (smax, pd * extent), (opac, min_op)):
        assert np.min(np.abs(q - lim) / lim) > 1e-5, "a decision sits on its threshold: pick other inputs"
    big = g >= thr
    split_ids = np.nonzero(big & (smax > pd * extent))[0]
    assert big.sum() > 100 and len(split_ids) > 50 and (big & (smax <= pd * extent)).sum() > 50
    assert (opac < min_op).sum() > 100
    dst = ctx.densify(scene, adam, torch.as_tensor(accum, device="cuda"), torch.as_tensor(denom, device="cuda"),
                      torch.as_tensor(normals, device="cuda"), extent, thr, pd, min_op)
    ctx.sync_status()
    W2, M2, V2, C2 = orc.densify(W, M, V, Cn, scene.step, hp, accum.astype(np.float64), denom.astype(np.float64),
                                 extent, normals[:, :, split_ids].astype(np.float64), thr, pd, min_op)
    assert dst.n == W2.shape[1] and dst.step == scene.step
    dm, dv = dst.moments()
    gw = dst.params().cpu().numpy().astype(np.float64)
    gm, gv = dm.cpu().numpy().astype(np.float64), dv.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(dst.counter[:dst.n].cpu().numpy(), C2)
    u = 2.0 ** -23
    rows_sh = np.arange(D)[:, None] >= 11
    rel = np.where(rows_sh, 2.0 ** -7 if bf16 else 8 * u, 8 * u)     # bf16: one ulp (stochastic rounding)
    # FP32 restore of the caught-up rows: one rounding of w and of the table x direction product
    for name, a, b in (("w", gw, W2), ("m", gm, M2), ("v", gv, V2)):
        bound = rel * np.abs(b) + (2e-6 if name == "w" else 1e-12) + (2.0 ** -7 * np.abs(b) if bf16 and name != "w" else 0)
        if bf16:
            # a bf16 store is a neighbour of its FP32 value: within one ulp of the larger magnitude
            mag = np.maximum(np.abs(a), np.abs(b)) + 1e-30
            ulp = 2.0 ** (np.floor(np.log2(mag)) - 7)
            bound = np.where(rows_sh, np.maximum(bound, ulp + 8 * u * np.abs(b) + (2e-6 if name == "w" else 1e-12)),
                             bound)
        err = np.abs(a - b)
        assert np.all(err <= bound), (name, float(np.max(err / bound)), np.unravel_index(np.argmax(err / bound), err.shape))
    # the geometry restore directions of the new scene are those of its stored moments
    rd = dst.rdir_geo[:, :dst.n].cpu().numpy().astype(np.float64)
    want = gm[:11] / (np.sqrt(gv[:11]) + 1e-15)
    np.testing.assert_allclose(rd, want, rtol=1e-5, atol=1e-30)
    print(f"densify ({prec_name}): {n} -> {dst.n} Gaussians, {len(split_ids)} split, "
          f"{int((big & (smax <= pd * extent)).sum())} cloned before pruning")


def test_densify_reports_a_small_destination(gs, orc):
    from paper_2509_15645_b300 import _lib
    ctx, scene, adam = _trained_scene(gs, orc, gs.GS_FP32, n=4000, steps=2)
    n = scene.n
    accum = torch.full((n,), 1.0, device="cuda")        # every Gaussian densifies: splits grow the scene
    denom = torch.ones(n, device="cuda")
    normals = torch.zeros(2, 3, n, device="cuda")
    dst = ctx.densify(scene, adam, accum, denom, normals, extent=1e-6, min_opacity=0.0, capacity=n // 2)
    ctx.sync_status()
    assert dst.n == 2 * n                                  # retried with the size the first call reported
