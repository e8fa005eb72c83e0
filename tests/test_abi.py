"""The C-ABI library loads and exports every entry point the header declares;
host-side argument checks work without a GPU (no compute calls here)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names += re.findall(r"GS_API\s+[\w\s\*]+?\b(gs_\w+)\s*\(", open(h).read())
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_15645_b300 import _lib
    from paper_2509_15645_b300 import build
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2509_15645_b300 import _lib
    assert set(names) == set(_lib.EXPORTS), set(names) ^ set(_lib.EXPORTS)


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and offsets."""
    import subprocess
    from paper_2509_15645_b300 import _lib
    structs = {"gs_camera": _lib.Camera, "gs_scene": _lib.Scene, "gs_adam_cfg": _lib.AdamCfg, "gs_config": _lib.Config}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs_b300.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def _cfg(**kw):
    from paper_2509_15645_b300 import _lib
    c = _lib.Config()
    d = dict(max_gaussians=10_000_000, max_visible=4_000_000, max_keys=40_000_000, max_width=1920,
             max_height=1080, tile_w=16, tile_h=16, max_views=4, max_sh_degree=3)
    d.update(kw)
    for k, v in d.items():
        setattr(c, k, v)
    return c


def test_workspace_size_and_validation(lib):
    from paper_2509_15645_b300 import _lib
    nb = C.c_size_t(0)
    assert lib.gs_workspace_size(C.byref(_cfg()), C.byref(nb)) == _lib.GS_OK
    assert nb.value > 59 * 4_000_000 * 4          # at least the compact parameter planes
    small = C.c_size_t(0)
    lib.gs_workspace_size(C.byref(_cfg(max_gaussians=1000, max_visible=1000, max_keys=10000, max_views=1)),
                          C.byref(small))
    assert 0 < small.value < nb.value
    for bad in (dict(tile_w=10), dict(max_views=0), dict(max_views=9), dict(max_sh_degree=4),
                dict(max_gaussians=0), dict(max_width=0), dict(max_keys=0)):
        assert lib.gs_workspace_size(C.byref(_cfg(**bad)), C.byref(nb)) == _lib.GS_ERR_INVALID_ARG, bad


def test_null_context_is_rejected(lib):
    from paper_2509_15645_b300 import _lib
    sc, cam, ad = _lib.Scene(), _lib.Camera(), _lib.AdamCfg()
    z = C.c_void_p(0)
    assert lib.gs_cull(None, C.byref(sc), C.byref(cam), None, z, z, z) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_render_fwd(None, C.byref(sc), C.byref(cam), None, z, z, z, z) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_render_bwd(None, z, z, 1, z) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_adam_deferred(None, C.byref(sc), z, z, z, 1, C.byref(ad), z) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_step(None, C.byref(sc), C.byref(cam), None, 1, C.byref(ad), z, z) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_destroy(None) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_last_error(None) == b"null context"
    c = _cfg()
    h = C.c_void_p()
    c.tile_w = 7
    assert lib.gs_create(C.byref(h), C.byref(c), 0, None, 0) == _lib.GS_ERR_INVALID_ARG


def test_staging_ring_configuration(lib):
    """The host tier's staging ring: its size follows stage_chunks, the chunk
    size and the element size of the staged rows (w, m, v of the 48 SH planes
    at degree 3); out-of-range chunk shifts and element sizes are refused, and
    the 32-pixel tiles of the warp-tile rasterizer are accepted."""
    from paper_2509_15645_b300 import _lib

    def size(**kw):
        nb = C.c_size_t(0)
        st = lib.gs_workspace_size(C.byref(_cfg(**kw)), C.byref(nb))
        return st, nb.value

    st0, base = size()
    assert st0 == _lib.GS_OK
    st, ring4 = size(stage_chunks=100, chunk_shift=11)
    assert st == _lib.GS_OK
    st, ring2 = size(stage_chunks=100, chunk_shift=11, stage_elem_bytes=2)
    assert st == _lib.GS_OK
    planes = 48
    # the ring (3 arrays) plus chunk tables; allocations are 256-byte aligned
    assert abs((ring4 - base) - 3 * planes * (100 << 11) * 4) < 4096 + 8 * (10_000_000 >> 11)
    assert abs((ring2 - base) - 3 * planes * (100 << 11) * 2) < 4096 + 8 * (10_000_000 >> 11)
    assert size(stage_chunks=100, chunk_shift=13)[1] > ring4
    for bad in (dict(stage_chunks=10, chunk_shift=9), dict(stage_chunks=10, chunk_shift=21),
                dict(stage_chunks=10, stage_elem_bytes=3), dict(stage_chunks=-1), dict(tile_w=32, tile_h=16)):
        assert size(**bad)[0] == _lib.GS_ERR_INVALID_ARG, bad
    for good in (dict(tile_w=8, tile_h=4), dict(tile_w=4, tile_h=8), dict(tile_w=64, tile_h=4)):
        assert size(**good)[0] == _lib.GS_OK, good


def test_region_cameras_marshal_the_full_image():
    """split_regions tiles the view; each region's struct carries the view's
    intrinsics (the library moves the principal point), its origin and the
    full image size; a whole-image camera leaves the region fields at 0."""
    import numpy as np
    import torch
    from paper_2509_15645_b300 import api
    from synth import scenes
    cam = scenes.camera_lookat((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 120, 80, 60.0, up=(0, -1, 0))
    whole = api.camera_struct(cam)
    assert (whole.x0, whole.y0, whole.full_width, whole.full_height) == (0, 0, 0, 0)
    img = torch.arange(3 * 80 * 120, dtype=torch.float32).view(3, 80, 120)
    for axis, split in ((0, 48), (1, 32)):
        regs = api.split_regions(cam, axis, split)
        area = 0
        for r in regs:
            cs = api.camera_struct(r)
            assert (cs.full_width, cs.full_height) == (120, 80)
            assert (cs.x0, cs.y0, cs.width, cs.height) == (r.x0, r.y0, r.width, r.height)
            assert cs.cx == whole.cx and cs.cy == whole.cy and cs.fx == whole.fx
            crop = r.crop(img)
            assert crop.is_contiguous() and tuple(crop.shape) == (3, r.height, r.width)
            assert torch.equal(crop, img[:, r.y0:r.y0 + r.height, r.x0:r.x0 + r.width])
            area += r.width * r.height
        assert area == 120 * 80
        assert (regs[1].x0, regs[1].y0) == ((split, 0) if axis == 0 else (0, split))
    assert np.all(np.asarray(regs[0].R) == np.asarray(cam.R))


def test_noalloc_cull_rejects_before_any_launch(lib):
    """gs_cull_noalloc refuses what gs_cull refuses, on the host, before any
    CUDA call (so this runs without a GPU): an oversize scene, an SH degree
    outside 0..3, a non-finite focal length, unusable Adam hyper-parameters."""

    def scene(n=1000, deg=1):
        sc = _lib.Scene()
        sc.n, sc.pitch, sc.sh_degree = n, (n + 3) // 4 * 4, deg
        sc.geo = 256                                 # never dereferenced: rejected on the host first
        return sc

    def cam(fx=50.0):
        c = _lib.Camera()
        c.width, c.height, c.fx, c.fy, c.near_z, c.far_z = 64, 64, fx, 50.0, 0.01, 100.0
        return c

    from paper_2509_15645_b300 import _lib
    z = C.c_void_p(256)
    call = lambda sc, cm, ad=None: lib.gs_cull_noalloc(C.byref(sc), C.byref(cm), C.byref(ad) if ad else None, 16, 16,
                                                       z, z, None, None)
    assert call(scene(n=(1 << 24) + 1), cam()) == _lib.GS_ERR_CAPACITY
    assert call(scene(deg=4), cam()) == _lib.GS_ERR_INVALID_ARG
    assert call(scene(deg=-1), cam()) == _lib.GS_ERR_INVALID_ARG
    assert call(scene(), cam(fx=float("inf"))) == _lib.GS_ERR_INVALID_ARG
    assert call(scene(), cam(fx=float("nan"))) == _lib.GS_ERR_INVALID_ARG
    from paper_2509_15645_b300 import api
    for bad in (dict(beta2=1.0), dict(beta1=-0.1), dict(eps=-1.0), dict(max_defer=16), dict(max_defer=0),
                dict(mode=7)):
        assert call(scene(), cam(), api.adam_struct(**bad)) == _lib.GS_ERR_INVALID_ARG, bad


def test_render_rounds_bound_the_workspace(lib):
    """gs_config.render_views: render buffers for that many views only (the
    per-view cull buffers stay for max_views), so two regions rendered one
    after the other need less workspace than two at once; values outside
    0..max_views are refused."""
    from paper_2509_15645_b300 import api
    kw = dict(max_gaussians=1_000_000, max_visible=400_000, max_keys=8_000_000, max_width=1920, max_height=1080,
              tile=(8, 4), max_views=2, max_sh_degree=3)
    both = api.Context.workspace_bytes(**kw)
    one = api.Context.workspace_bytes(**kw, render_views=1)
    single = api.Context.workspace_bytes(**dict(kw, max_views=1))
    assert api.Context.workspace_bytes(**kw, render_views=2) == both
    assert one < both and both - one > 0.4 * (both - single)
    from paper_2509_15645_b300 import _lib
    for bad in (3, -1):
        with pytest.raises(_lib.GsError):
            api.Context.workspace_bytes(**kw, render_views=bad)
    # list-order records: 3 float4 per key of capacity and view
    assert api.Context.workspace_bytes(**kw, list_records=1) - both >= 2 * 48 * kw["max_keys"]
    with pytest.raises(_lib.GsError):
        api.Context.workspace_bytes(**kw, list_records=2)
