"""gs_cull_noalloc: the frustum cull for callers that cannot allocate device
memory (a framework whose memory pool owns every device byte, loops that
forbid allocation after start-up, callers that need a fixed footprint).  It
must give exactly what gs_cull on a context gives, call after call, through
the C ABI.  This file sorts last so that a run stopping at its first failure
has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import scenes

pytestmark = pytest.mark.gpu


def _noalloc(lib, _lib, scene, cam_s, adam, tile, ids, nv, status=None):
    return lib.gs_cull_noalloc(C.byref(scene.struct()), C.byref(cam_s), C.byref(adam) if adam is not None else None,
                               tile[0], tile[1], C.c_void_p(ids.data_ptr()), C.c_void_p(nv.data_ptr()),
                               C.c_void_p(status.data_ptr() if status is not None else 0),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_cull_matches_context_cull_twice():
    assert torch.cuda.is_available()
    import paper_2509_15645_b300 as gs
    from paper_2509_15645_b300 import _lib
    lib = _lib.load()
    n, deg, tile = 20_000, 1, (16, 16)
    P = scenes.uniform_cube_scene(n, seed=21, sh_degree=deg, log_scale_mean=-3.0)
    P[0:3] *= 2.0                                   # part of the cube outside the views
    scene = gs.GaussianScene(P, deg)
    rng = np.random.default_rng(0)
    scene.m[:, :n] = torch.as_tensor(rng.normal(size=(scene.D, n)) * 1e-3, dtype=torch.float32, device="cuda")
    scene.v[:, :n] = torch.as_tensor(rng.uniform(1e-8, 1e-6, (scene.D, n)), dtype=torch.float32, device="cuda")
    scene.counter[:n] = torch.as_tensor(rng.integers(0, 16, n), dtype=torch.uint8, device="cuda")
    scene.step = 40
    adam = gs.adam_struct(lr=1e-2, eps=1e-15)
    cams = [scenes.camera_lookat((0.2, -0.1, -3.0), (0.0, 0.0, 0.0), 77, 45, 60.0, up=(0, -1, 0)),
            scenes.camera_lookat((-1.5, 0.4, -2.5), (0.3, 0.0, 0.5), 128, 96, 75.0, up=(0, -1, 0))]
    ctx = gs.Context(max_gaussians=n, max_visible=n, max_keys=10 * n, max_width=128, max_height=96, tile=tile,
                     max_sh_degree=deg)
    ctx.refresh_rdir(scene, adam)                    # m and v were set directly
    for cam, ad in ((cams[0], None), (cams[1], adam)):           # two calls in a row, the second with restore
        ids_ref, nv_ref = ctx.cull(scene, cam, ad)
        ids = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        nv = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        st = _noalloc(lib, _lib, scene, gs.camera_struct(cam), ad, tile, ids, nv, status)
        assert st == _lib.GS_OK
        ctx.sync_status()
        k = int(nv_ref.item())
        assert 0 < k < n
        assert int(status.item()) == _lib.GS_OK
        assert int(nv.item()) == k
        assert torch.equal(ids[:k], ids_ref[:k])


def test_noalloc_cull_reports_a_timeout_and_recovers():
    """A cull block that gives up waiting for its own copies (the first-wait
    limit set to 0: every block gives up at once, then lets its copies land)
    is reported through the status word, with no visible Gaussian; with the
    default limit restored the next call gives gs_cull's result again."""
    assert torch.cuda.is_available()
    import paper_2509_15645_b300 as gs
    from paper_2509_15645_b300 import _lib
    lib = _lib.load()
    n, deg, tile = 20_000, 0, (16, 16)
    P = scenes.uniform_cube_scene(n, seed=22, sh_degree=deg, log_scale_mean=-3.0)
    scene = gs.GaussianScene(P, deg)
    cam = scenes.camera_lookat((0.2, -0.1, -3.0), (0.0, 0.0, 0.0), 77, 45, 60.0, up=(0, -1, 0))
    ctx = gs.Context(max_gaussians=n, max_visible=n, max_keys=10 * n, max_width=77, max_height=45, tile=tile,
                     max_sh_degree=deg)
    ids_ref, nv_ref = ctx.cull(scene, cam)
    ctx.sync_status()
    ids = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    nv = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert lib.gs_set_cull_wait_limit(None, 0) == _lib.GS_OK
    try:
        assert _noalloc(lib, _lib, scene, gs.camera_struct(cam), None, tile, ids, nv, status) == _lib.GS_OK
        torch.cuda.synchronize()
        assert int(status.item()) == _lib.GS_ERR_TIMEOUT
        assert int(nv.item()) == 0
    finally:
        assert lib.gs_set_cull_wait_limit(None, 1 << 24) == _lib.GS_OK
    assert _noalloc(lib, _lib, scene, gs.camera_struct(cam), None, tile, ids, nv, status) == _lib.GS_OK
    torch.cuda.synchronize()
    k = int(nv_ref.item())
    assert int(status.item()) == _lib.GS_OK and int(nv.item()) == k
    assert torch.equal(ids[:k], ids_ref[:k])
