"""Host tier (selective offloading, §4.2): SH planes with their moments and
restore directions in pinned host memory, streamed chunk by chunk through the
context's staging ring by gs_step.  The arithmetic is the same as for a
device-resident scene; the only run-to-run difference is the order of the
rasterizer's atomic gradient sums (a few FP32 ulps).  With eps = 1 the Adam
step is close to linear in the gradient (no sign(g) amplification of those
ulps), so after a run long enough for never-visible Gaussians to reach the
counter bound (their chunks staged for the optimizer alone) every stored value
must agree to a few ulps of its storage type, while a staging fault (a wrong
row, a lost write-back) would move values by the whole update."""
import numpy as np
import pytest
import torch

from helpers import cam_f32
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available()
    import paper_2509_15645_b300 as gs
    return gs


def _views():
    # nadir-oblique views of parts of a heightfield: each sees 7-11 of the 40
    # chunks of 1024 Gaussians, so most chunks stay on the host for many steps
    return [cam_f32(scenes.camera_aerial((50 * np.cos(a), 50 * np.sin(a), 40.0), a, -np.pi / 2 + 0.3, 96, 72, 50.0))
            for a in np.linspace(0, 2 * np.pi, 5)[:4]]


def _scene(n, deg, seed):
    return scenes.heightfield_scene(n, seed=seed, half_extent=100.0, amplitude=5.0, wavelength=(20.0, 25.0),
                                    n_clusters=2, cluster_size=2000, sh_degree=deg)


def _run(gs, P, deg, prec, tier, steps, n_views=1, stage_chunks=64, shift=10, ring_eb=None):
    n = P.shape[1]
    cams = _views()
    if ring_eb is None:      # bf16 scenes stage through a ring of 2-byte rows
        ring_eb = 4 if prec == gs.GS_FP32 else 2
    ctx = gs.Context(max_gaussians=n, max_visible=n, max_keys=64 * n, max_width=96, max_height=72, tile=(8, 8),
                     max_views=2, max_sh_degree=deg, stage_chunks=stage_chunks if tier else 0, chunk_shift=shift,
                     stage_elem_bytes=ring_eb if tier else 0)
    tgt = [torch.full((3, 72, 96), 0.3 + 0.1 * k, device="cuda") for k in range(len(cams))]
    scene = gs.GaussianScene(P, deg, precision=prec, tier=tier)
    adam = gs.adam_struct(lr=[1e-3, 1e-2, 1e-2, 1.0, 10.0, 10.0], eps=1.0, seed=5)
    staged = []
    for t in range(steps):
        vs = [(t + j) % len(cams) for j in range(n_views)]
        ctx.step(scene, [cams[v] for v in vs], [tgt[v] for v in vs], adam)
        if tier:
            staged.append(ctx.host_tier_stats()[0])
    if tier:     # the stream waits for the write-backs; only the stream is synchronised
        ctx.wait_copies()
        torch.cuda.current_stream().synchronize()
    else:
        ctx.sync_status()
    m, v = scene.moments()
    out = dict(w=scene.params().cpu().numpy(), m=m.cpu().numpy(), v=v.cpu().numpy(),
               counter=scene.counter[:n].cpu().numpy(), staged=staged)
    ctx.sync_status()
    return out


@pytest.mark.parametrize("prec_name,n_views,ring", [("GS_FP32", 1, 64), ("GS_BF16_SH_MOM", 1, 16), ("GS_FP32", 2, 24),
                                                    ("GS_FP32", 1, 13)])
def test_host_tier_matches_resident(gs, prec_name, n_views, ring):
    """ring: staging slots; below the 40 chunks the counter-bound steps stage
    their optimizer-only chunks in several rounds."""
    prec = getattr(gs, prec_name)
    n, deg, steps = 40_000, 3, 20
    P = _scene(n, deg, 31)
    a = _run(gs, P, deg, prec, gs.GS_TIER_DEVICE, steps, n_views)
    b = _run(gs, P, deg, prec, gs.GS_TIER_HOST_SH, steps, n_views, stage_chunks=ring)
    nch = (n + 1023) // 1024
    assert all(0 < k <= nch for k in b["staged"])
    assert min(b["staged"]) < nch                       # some steps leave chunks on the host
    if ring < nch:
        assert max(b["staged"]) > ring                  # a counter-bound step staged in several rounds
    assert np.mean(a["counter"] != b["counter"]) <= 1e-3
    # storage ulp: 2^-23 (fp32) or 2^-7 (bf16, stochastic rounding may pick the other neighbour)
    ulp = 2.0 ** -23 if prec == gs.GS_FP32 else 2.0 ** -7
    for k in ("w", "m", "v"):
        x, y = a[k], b[k]
        scale = np.abs(x).max(axis=1, keepdims=True) + 1e-30
        if k == "w":                                    # geometry stays fp32 in every form
            bound = np.where(np.arange(x.shape[0])[:, None] < 11, 4 * 2.0 ** -23 * np.abs(x),
                             4 * ulp * np.abs(x)) + 1e-7
        else:
            bound = 4 * ulp * np.abs(x) + 1e-4 * scale
        assert np.all(np.abs(x - y) <= bound), (k, np.max(np.abs(x - y) / bound))
    # the SH rows trained and came back from the device
    w0 = torch.as_tensor(P[11:]).to(torch.float32 if prec == gs.GS_FP32 else torch.bfloat16).float().numpy()
    assert np.mean(b["w"][11:] != w0) > 0.03           # (the Gaussians the views saw)


def test_host_tier_reports_a_small_ring(gs):
    from paper_2509_15645_b300 import _lib
    n, deg = 40_000, 1
    P = _scene(n, deg, 32)
    with pytest.raises(_lib.GsError) as e:       # a view's visible chunks alone exceed the ring
        _run(gs, P, deg, gs.GS_FP32, gs.GS_TIER_HOST_SH, 1, stage_chunks=2)
    assert e.value.status == _lib.GS_ERR_CAPACITY


def test_host_tier_refuses_fp32_rows_in_a_bf16_ring(gs):
    from paper_2509_15645_b300 import _lib
    n, deg = 40_000, 1
    P = _scene(n, deg, 33)
    with pytest.raises(_lib.GsError) as e:
        _run(gs, P, deg, gs.GS_FP32, gs.GS_TIER_HOST_SH, 1, ring_eb=2)
    assert e.value.status == _lib.GS_ERR_INVALID_ARG
