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


def _noalloc(lib, _lib, scene, cam_s, adam, tile, ids, nv):
    return lib.gs_cull_noalloc(C.byref(scene.struct()), C.byref(cam_s), C.byref(adam) if adam is not None else None,
                               tile[0], tile[1], C.c_void_p(ids.data_ptr()), C.c_void_p(nv.data_ptr()),
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
        st = _noalloc(lib, _lib, scene, gs.camera_struct(cam), ad, tile, ids, nv)
        assert st == _lib.GS_OK
        ctx.sync_status()
        k = int(nv_ref.item())
        assert 0 < k < n
        assert int(nv.item()) == k
        assert torch.equal(ids[:k], ids_ref[:k])


def test_noalloc_cull_rejects_oversize_scene():
    from paper_2509_15645_b300 import _lib
    lib = _lib.load()
    sc = _lib.Scene()
    sc.n = (1 << 24) + 1
    sc.pitch = (1 << 24) + 4
    sc.geo = 256                                     # never dereferenced: the size check comes first
    cam = _lib.Camera()
    cam.width, cam.height, cam.fx, cam.fy, cam.near_z, cam.far_z = 64, 64, 50.0, 50.0, 0.01, 100.0
    z = C.c_void_p(256)
    assert lib.gs_cull_noalloc(C.byref(sc), C.byref(cam), None, 16, 16, z, z, None) == _lib.GS_ERR_CAPACITY
