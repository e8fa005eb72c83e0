"""Torch-facing wrappers of the C ABI.

PyTorch supplies device memory and streams only; every step of the hot path
runs in the CUDA library.  Layouts follow include/gs_b300.h: parameters are
[D][pitch] float32 planes (geometry rows 0..10, SH rows 11..), compact
per-visible arrays are [D][cap].
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


def n_params(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class _DeviceArray:
    """Exposes a raw device array (int32 unless typestr says otherwise) to torch
    through __cuda_array_interface__."""

    def __init__(self, ptr, n, typestr="<i4"):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False), "version": 3}


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def camera_struct(cam) -> L.Camera:
    """From any object with R (3x3), t (3), fx, fy, cx, cy, width, height,
    near, far (e.g. ``synth.scenes.Camera``)."""
    c = L.Camera()
    R = [float(x) for row in cam.R for x in row]
    for k in range(9):
        c.R[k] = R[k]
    for k in range(3):
        c.t[k] = float(cam.t[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_z, c.far_z = float(getattr(cam, "near", 0.01)), float(getattr(cam, "far", 1e10))
    c.width, c.height = int(cam.width), int(cam.height)
    if getattr(cam, "full_width", 0):
        c.x0, c.y0 = int(cam.x0), int(cam.y0)
        c.full_width, c.full_height = int(cam.full_width), int(cam.full_height)
    return c


class RegionCamera:
    """Part of a view (§4.4 image splitting): the region [x0, x0 + width) x
    [y0, y0 + height) of ``cam``'s full image.  It culls, renders and steps like
    a camera; the projection's guard band and the L1 normalisation are the full
    image's, so the losses and gradients of a view's regions, summed, are the
    whole view's."""

    def __init__(self, cam, x0, y0, width, height):
        self.R, self.t = cam.R, cam.t
        self.fx, self.fy, self.cx, self.cy = cam.fx, cam.fy, cam.cx, cam.cy
        self.near, self.far = getattr(cam, "near", 0.01), getattr(cam, "far", 1e10)
        self.x0, self.y0, self.width, self.height = int(x0), int(y0), int(width), int(height)
        self.full_width, self.full_height = int(cam.width), int(cam.height)

    def crop(self, image):
        """This region of a full-view [3][H][W] image, as a contiguous tensor."""
        return image[:, self.y0:self.y0 + self.height, self.x0:self.x0 + self.width].contiguous()


def split_regions(cam, axis: int, split: int):
    """The two regions of ``cam`` split at pixel ``split``: axis 0 columns
    [0, split) and [split, W), axis 1 rows [0, split) and [split, H)."""
    W, H = int(cam.width), int(cam.height)
    if axis == 0:
        return [RegionCamera(cam, 0, 0, split, H), RegionCamera(cam, split, 0, W - split, H)]
    return [RegionCamera(cam, 0, 0, W, split), RegionCamera(cam, 0, split, W, H - split)]


def adam_struct(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-15, max_defer=15, mode=L.GS_ADAM_DEFERRED,
                seed=0, optimizer=L.GS_OPT_ADAM, weight_decay=0.0) -> L.AdamCfg:
    """Optimizer hyper-parameters.  optimizer GS_OPT_ADAM, GS_OPT_ADAMW
    (decoupled ``weight_decay``) or GS_OPT_SGDM (momentum ``beta1``)."""
    a = L.AdamCfg()
    lrs = [lr] * 6 if isinstance(lr, (int, float)) else list(lr)
    for k in range(6):
        a.lr[k] = float(lrs[k])
    a.beta1, a.beta2, a.eps, a.max_defer, a.mode, a.seed = beta1, beta2, eps, max_defer, mode, seed
    a.optimizer, a.weight_decay = int(optimizer), float(weight_decay)
    return a


def adam_tables(adam: L.AdamCfg, step: int) -> dict:
    """The deferred update's tables for optimizer step ``step`` as the kernels
    receive them (Fig. 10): ``param`` [6][16], ``mom`` [16], ``var`` [16],
    ``step_size`` [6], ``bias_corr``, ``decay`` [6][16].  Host only."""
    param, mom, var, ss, bc = (C.c_float * 96)(), (C.c_float * 16)(), (C.c_float * 16)(), (C.c_float * 6)(), C.c_float()
    dec = (C.c_float * 96)()
    st = L.load().gs_adam_tables(C.byref(adam), int(step), param, mom, var, ss, C.byref(bc), dec)
    if st != L.GS_OK:
        raise L.GsError(st, "gs_adam_tables")
    return {"param": [list(param[g * 16:(g + 1) * 16]) for g in range(6)], "mom": list(mom), "var": list(var),
            "step_size": list(ss), "bias_corr": bc.value, "decay": [list(dec[g * 16:(g + 1) * 16]) for g in range(6)]}


class GaussianScene:
    """A Gaussian set with its optimizer state.

    precision GS_FP32: ``w`` is one [D][pitch] float32 tensor (geometry planes
    then SH planes; ``geo`` and ``sh`` are views of it), m / v float32.  BF16
    forms: ``geo`` [11][pitch] float32 (master copy), ``sh`` [D-11][pitch]
    bfloat16, m / v bfloat16.  Both: ``rdir_geo`` [11][pitch] float32, the
    restore directions of the geometry planes the optimizer keeps.

    tier GS_TIER_HOST_SH: the geometry planes with their m, v (``m``, ``v``
    [11][pitch]) and ``rdir_geo`` stay on the device; the SH planes ``sh`` and
    their ``m_sh``, ``v_sh`` are pinned host tensors [D-11][pitch] that gs_step
    streams (read them after ``Context.sync_status``, or from work enqueued on a
    stream after ``Context.wait_copies``).  tier GS_TIER_HOST_CPU_OPT (fp32):
    the same, with ``sh``, ``m_sh``, ``v_sh`` one row per Gaussian,
    [pitch][D-11], stepped by the host cores (read them after
    ``Context.sync_status``)."""

    def __init__(self, params, sh_degree: int, device="cuda", with_optimizer=True, with_rdir=True,
                 precision=L.GS_FP32, tier=L.GS_TIER_DEVICE):
        D, n = params.shape
        assert D == n_params(sh_degree)
        self.n, self.sh_degree, self.D, self.precision, self.tier = n, sh_degree, D, precision, tier
        self.pitch = (n + 3) // 4 * 4
        P = self.pitch
        src = torch.as_tensor(params, dtype=torch.float32)
        mdtype = torch.float32 if precision == L.GS_FP32 else torch.bfloat16
        self.w = None
        self.m = self.v = self.counter = None
        self.m_sh = self.v_sh = None
        self.rdir_geo = None
        host = tier in (L.GS_TIER_HOST_SH, L.GS_TIER_HOST_CPU_OPT)
        if host:
            assert tier == L.GS_TIER_HOST_SH or precision == L.GS_FP32, "the host-core optimizer tier is fp32"
            assert with_optimizer, "the host tier holds optimizer state"
            pin = dict(device="cpu", pin_memory=True)
            self.geo = torch.zeros(11, P, dtype=torch.float32, device=device)
            self.geo[:, :n] = src[:11].to(device)
            self.m = torch.zeros(11, P, dtype=mdtype, device=device)
            self.v = torch.zeros(11, P, dtype=mdtype, device=device)
            if tier == L.GS_TIER_HOST_CPU_OPT:       # one row of SH values per Gaussian
                self.sh = torch.zeros(P, D - 11, dtype=mdtype, **pin)
                self.sh[:n] = src[11:].T.to(mdtype)
                self.m_sh = torch.zeros(P, D - 11, dtype=mdtype, **pin)
                self.v_sh = torch.zeros(P, D - 11, dtype=mdtype, **pin)
            else:
                self.sh = torch.zeros(D - 11, P, dtype=mdtype, **pin)
                self.sh[:, :n] = src[11:].to(mdtype)
                self.m_sh = torch.zeros(D - 11, P, dtype=mdtype, **pin)
                self.v_sh = torch.zeros(D - 11, P, dtype=mdtype, **pin)
            self.counter = torch.zeros(P, dtype=torch.uint8, device=device)
            if with_rdir:     # geometry directions only: the SH ones are recomputed on the device
                self.rdir_geo = torch.zeros(11, P, dtype=torch.float32, device=device)
            self.step = 0
            return
        src = src.to(device)
        if precision == L.GS_FP32:
            self.w = torch.zeros(D, P, dtype=torch.float32, device=device)
            self.w[:, :n] = src
            self.geo, self.sh = self.w[:11], self.w[11:]
        else:
            self.geo = torch.zeros(11, P, dtype=torch.float32, device=device)
            self.sh = torch.zeros(D - 11, P, dtype=torch.bfloat16, device=device)
            self.geo[:, :n] = src[:11]
            self.sh[:, :n] = src[11:].to(torch.bfloat16)
        if with_optimizer:
            self.m = torch.zeros(D, P, dtype=mdtype, device=device)
            self.v = torch.zeros(D, P, dtype=mdtype, device=device)
            self.counter = torch.zeros(P, dtype=torch.uint8, device=device)
            if with_rdir:
                # restore directions m / (sqrt(v) + eps) of the geometry planes, zero while m = v = 0
                self.rdir_geo = torch.zeros(11, P, dtype=torch.float32, device=device)
        self.step = 0

    def struct(self) -> L.Scene:
        s = L.Scene()
        s.n, s.pitch, s.sh_degree, s.precision, s.tier = self.n, self.pitch, self.sh_degree, self.precision, self.tier
        if self.w is not None:
            s.geo = self.w.data_ptr()
            s.sh = self.w.data_ptr() + 11 * self.pitch * 4
        else:
            s.geo = self.geo.data_ptr()
            s.sh = self.sh.data_ptr() if self.tier == L.GS_TIER_DEVICE else None
        s.m = self.m.data_ptr() if self.m is not None else None
        s.v = self.v.data_ptr() if self.v is not None else None
        s.rdir = self.rdir_geo.data_ptr() if self.rdir_geo is not None else None
        s.counter = self.counter.data_ptr() if self.counter is not None else None
        if self.tier != L.GS_TIER_DEVICE:
            s.host_sh, s.host_m, s.host_v = self.sh.data_ptr(), self.m_sh.data_ptr(), self.v_sh.data_ptr()
            s.host_rdir = None
        s.step = self.step
        return s

    def _sh_planes(self, t):
        """[D-11][n] view of SH planes (host rows of the CPU-optimizer tier transposed)."""
        return t[:self.n].T if self.tier == L.GS_TIER_HOST_CPU_OPT else t[:, :self.n]

    def params(self):
        """Stored parameters as float32 [D][n] on the geometry's device."""
        if self.w is not None:
            return self.w[:, :self.n]
        return torch.cat([self.geo[:, :self.n], self._sh_planes(self.sh).to(self.geo.device).float()])

    def moments(self):
        """(m, v) as float32 [D][n] on the geometry's device."""
        if self.tier != L.GS_TIER_DEVICE:
            dev = self.geo.device
            return (torch.cat([self.m[:, :self.n].float(), self._sh_planes(self.m_sh).to(dev).float()]),
                    torch.cat([self.v[:, :self.n].float(), self._sh_planes(self.v_sh).to(dev).float()]))
        return self.m[:, :self.n].float(), self.v[:, :self.n].float()


class Context:
    """One gs_ctx: scratch workspace (a torch allocation) and the hot-path calls."""

    def __init__(self, max_gaussians, max_visible, max_keys, max_width, max_height, tile=(8, 8), max_views=1,
                 max_sh_degree=3, device=0, stage_chunks=0, chunk_shift=0, stage_elem_bytes=0, render_views=0,
                 list_records=0, cpu_opt=0):
        self.lib = L.load()
        cfg = self._config(max_gaussians, max_visible, max_keys, max_width, max_height, tile, max_views,
                           max_sh_degree, stage_chunks, chunk_shift, stage_elem_bytes, render_views, list_records,
                           cpu_opt)
        self.cfg = cfg
        nb = C.c_size_t(0)
        self._check(self.lib.gs_workspace_size(C.byref(cfg), C.byref(nb)), "workspace size")
        self.device = torch.device("cuda", device)
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        self._check(self.lib.gs_create(C.byref(h), C.byref(cfg), device, _ptr(self.workspace), nb.value), "create")
        self.h = h
        self.max_visible = int(max_visible)

    @staticmethod
    def _config(max_gaussians, max_visible, max_keys, max_width, max_height, tile=(8, 8), max_views=1,
                max_sh_degree=3, stage_chunks=0, chunk_shift=0, stage_elem_bytes=0, render_views=0,
                list_records=0, cpu_opt=0):
        cfg = L.Config()
        cfg.cpu_opt = int(cpu_opt)
        cfg.render_views = int(render_views)
        cfg.list_records = int(list_records)
        cfg.stage_chunks, cfg.chunk_shift = int(stage_chunks), int(chunk_shift)
        cfg.stage_elem_bytes = int(stage_elem_bytes)
        cfg.max_gaussians, cfg.max_visible, cfg.max_keys = int(max_gaussians), int(max_visible), int(max_keys)
        cfg.max_width, cfg.max_height = int(max_width), int(max_height)
        cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
        cfg.max_views, cfg.max_sh_degree = int(max_views), int(max_sh_degree)
        return cfg

    @staticmethod
    def workspace_bytes(**kw):
        """Device workspace a context with these arguments would take."""
        cfg = Context._config(**kw)
        nb = C.c_size_t(0)
        st = L.load().gs_workspace_size(C.byref(cfg), C.byref(nb))
        if st != L.GS_OK:
            raise L.GsError(st, "workspace size")
        return nb.value

    def _check(self, st, what=""):
        if st != L.GS_OK:
            msg = self.lib.gs_last_error(self.h).decode() if getattr(self, "h", None) else what
            raise L.GsError(st, f"{what}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def sync_status(self, stream=None):
        st = self.lib.gs_sync_status(self.h, _stream(stream))
        self._check(st, "device status")

    def wait_copies(self, stream=None):
        """The stream waits for the host tier's write-backs still in flight."""
        self._check(self.lib.gs_wait_copies(self.h, _stream(stream)), "gs_wait_copies")

    def counters(self):
        """The context's device counters (a torch view, no copy): [0] visible
        count of the last cull, [1] keys of the last render, [2] update-set size
        of the last deferred Adam step, [3] latched status, [6] Gaussians of
        the last render projected through the FP64 covariance chain."""
        p = self.lib.gs_device_counters(self.h)
        return torch.as_tensor(_DeviceArray(p, 8), device=self.device)

    def render_lists(self, tiles):
        """Sorted (tile, compact index) keys and tile ranges of the last render
        (torch views of context memory)."""
        kt, kv, nk, rg = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
        self._check(self.lib.gs_render_lists(self.h, C.byref(kt), C.byref(kv), C.byref(nk), C.byref(rg)), "lists")
        n = int(torch.as_tensor(_DeviceArray(nk.value, 1), device=self.device).item())
        keys = torch.as_tensor(_DeviceArray(kt.value, max(n, 1)), device=self.device)[:n]
        vals = torch.as_tensor(_DeviceArray(kv.value, max(n, 1)), device=self.device)[:n]
        ranges = torch.as_tensor(_DeviceArray(rg.value, 2 * tiles), device=self.device).view(tiles, 2)
        return keys, vals, ranges

    def host_tier_stats(self):
        """(chunks staged, bytes moved host<->device) by the last host-tier gs_step."""
        ch, by = C.c_int64(0), C.c_int64(0)
        self._check(self.lib.gs_host_tier_stats(self.h, C.byref(ch), C.byref(by)), "host tier stats")
        return ch.value, by.value

    def set_cpu_threads(self, threads):
        """OpenMP threads of the host-core optimizer (GS_TIER_HOST_CPU_OPT; <= 0: every core)."""
        self._check(self.lib.gs_set_cpu_threads(self.h, int(threads)), "gs_set_cpu_threads")

    def cpu_tier_stats(self):
        """The last GS_TIER_HOST_CPU_OPT step: host ms forwarding, host ms of the
        worker's update, ms the step waited for the worker, bytes to / from the
        device, rows forwarded, members held for the next step."""
        out = (C.c_double * 7)()
        self._check(self.lib.gs_cpu_tier_stats(self.h, out), "gs_cpu_tier_stats")
        keys = ("forward_ms", "update_ms", "wait_ms", "h2d_bytes", "d2h_bytes", "rows", "held_members")
        return dict(zip(keys, list(out)))

    def step_gradients(self, D):
        """(ids int32 [n], gradients float32 [D][n]) the last gs_step's optimizer
        used (torch views of context memory, valid until the next render)."""
        g, p, i, nv = C.c_void_p(), C.c_int64(0), C.c_void_p(), C.c_void_p()
        self._check(self.lib.gs_step_gradients(self.h, C.byref(g), C.byref(p), C.byref(i), C.byref(nv)),
                    "gs_step_gradients")
        n = int(torch.as_tensor(_DeviceArray(nv.value, 1), device=self.device).item())
        ids = torch.as_tensor(_DeviceArray(i.value, max(n, 1)), device=self.device)[:n]
        grad = torch.as_tensor(_DeviceArray(g.value, D * p.value, "<f4"), device=self.device).view(D, p.value)[:, :n]
        return ids, grad

    def render_splats(self):
        """Projected splats of the last render, float32 [n_vis][4] each (torch
        views of context memory): (mean2d x, mean2d y, radius, opacity) and
        (conic A, B, C, depth)."""
        g, c, nv = C.c_void_p(), C.c_void_p(), C.c_void_p()
        self._check(self.lib.gs_render_splats(self.h, C.byref(g), C.byref(c), C.byref(nv)), "splats")
        n = int(torch.as_tensor(_DeviceArray(nv.value, 1), device=self.device).item())
        geom = torch.as_tensor(_DeviceArray(g.value, 4 * max(n, 1), "<f4"), device=self.device)[:4 * n].view(n, 4)
        conic = torch.as_tensor(_DeviceArray(c.value, 4 * max(n, 1), "<f4"), device=self.device)[:4 * n].view(n, 4)
        return geom, conic

    def cull(self, scene: GaussianScene, cam, adam=None, stream=None):
        ids = torch.empty(self.max_visible, dtype=torch.int32, device=self.device)
        n_vis = torch.zeros(1, dtype=torch.int32, device=self.device)
        sc = scene.struct()
        cs = camera_struct(cam)
        st = self.lib.gs_cull(self.h, C.byref(sc), C.byref(cs), C.byref(adam) if adam is not None else None,
                              _ptr(ids), _ptr(n_vis), _stream(stream))
        self._check(st, "gs_cull")
        return ids, n_vis

    def split_point(self, scene: GaussianScene, cam, adam=None, axis=None, steps=5, stream=None):
        """Balance-aware split of one view (§4.4, gs_split_point): returns
        (axis, split in pixels, (visible count of region 0, of region 1)).
        axis None: split across the longer image side."""
        if axis is None:
            axis = 0 if int(cam.width) >= int(cam.height) else 1
        sc = scene.struct()
        cs = camera_struct(cam)
        sp, cnt = C.c_int32(0), (C.c_int64 * 2)()
        st = self.lib.gs_split_point(self.h, C.byref(sc), C.byref(cs), C.byref(adam) if adam is not None else None,
                                     int(axis), int(steps), C.byref(sp), cnt, _stream(stream))
        self._check(st, "gs_split_point")
        return axis, sp.value, (cnt[0], cnt[1])

    def plan_split(self, scene: GaussianScene, cam, adam=None, mem_limit=0.3, axis=None, steps=5, stream=None):
        """§4.4: a view whose visible fraction of the scene exceeds
        ``mem_limit`` is trained as two regions.  Returns None (train the view
        whole) or the two RegionCamera objects of its balance-aware split."""
        _, n_vis = self.cull(scene, cam, adam, stream)
        if int(n_vis.item()) <= mem_limit * scene.n:
            return None
        ax, sp, _ = self.split_point(scene, cam, adam, axis, steps, stream)
        return split_regions(cam, ax, sp)

    def render_fwd(self, scene: GaussianScene, cam, ids, n_vis, adam=None, stream=None):
        img = torch.empty(3, int(cam.height), int(cam.width), dtype=torch.float32, device=self.device)
        sc = scene.struct()
        cs = camera_struct(cam)
        st = self.lib.gs_render_fwd(self.h, C.byref(sc), C.byref(cs), C.byref(adam) if adam is not None else None,
                                    _ptr(ids), _ptr(n_vis), _ptr(img), _stream(stream))
        self._check(st, "gs_render_fwd")
        return img

    def render_bwd(self, dimage, D, cap=None, stream=None):
        cap = cap or self.max_visible
        g = torch.empty(D, cap, dtype=torch.float32, device=self.device)
        st = self.lib.gs_render_bwd(self.h, _ptr(dimage.contiguous()), _ptr(g), cap, _stream(stream))
        self._check(st, "gs_render_bwd")
        return g

    def loss_l1(self, image, target, stream=None):
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        dimg = torch.empty_like(image)
        st = self.lib.gs_loss_l1(self.h, _ptr(image), _ptr(target), image.numel(), _ptr(loss), _ptr(dimg),
                                 _stream(stream))
        self._check(st, "gs_loss_l1")
        return loss, dimg

    def adam_deferred(self, scene: GaussianScene, ids, n_vis, grad_compact, adam, stream=None):
        sc = scene.struct()
        st = self.lib.gs_adam_deferred(self.h, C.byref(sc), _ptr(ids), _ptr(n_vis), _ptr(grad_compact),
                                       grad_compact.shape[1], C.byref(adam), _stream(stream))
        self._check(st, "gs_adam_deferred")
        scene.step = sc.step

    def refresh_rdir(self, scene: GaussianScene, adam, stream=None):
        """Recompute the restore directions after m or v were set directly."""
        sc = scene.struct()
        self._check(self.lib.gs_refresh_rdir(self.h, C.byref(sc), C.byref(adam), _stream(stream)), "gs_refresh_rdir")

    def materialize(self, scene: GaussianScene, adam, stream=None):
        w, m, v = (torch.empty(scene.D, scene.pitch, dtype=torch.float32, device=self.device) for _ in range(3))
        sc = scene.struct()
        st = self.lib.gs_adam_materialize(self.h, C.byref(sc), C.byref(adam), _ptr(w), _ptr(m), _ptr(v),
                                          _stream(stream))
        self._check(st, "gs_adam_materialize")
        return w, m, v

    def grad_scatter(self, scene: GaussianScene, ids, n_vis, grad_compact, stream=None):
        full = torch.empty(scene.D, scene.pitch, dtype=torch.float32, device=self.device)
        sc = scene.struct()
        st = self.lib.gs_grad_scatter(self.h, C.byref(sc), _ptr(ids), _ptr(n_vis), _ptr(grad_compact),
                                      grad_compact.shape[1], _ptr(full), _stream(stream))
        self._check(st, "gs_grad_scatter")
        return full

    def autotune(self, scene: GaussianScene, cam, stream=None):
        """Time the rasterizer variants on this scene and view; keep the fastest
        forward and backward.  Returns ((forward variant, backward variant),
        per-variant forward ms, per-variant backward ms; None where not allowed)."""
        chosen = (C.c_int32 * 2)(-1, -1)
        ms = (C.c_float * (2 * L.RASTER_VARIANTS))()
        sc = scene.struct()
        cs = camera_struct(cam)
        self._check(self.lib.gs_autotune(self.h, C.byref(sc), C.byref(cs), chosen, ms, _stream(stream)),
                    "gs_autotune")
        V = L.RASTER_VARIANTS
        conv = [None if t < 0 else t for t in ms]
        return (chosen[0], chosen[1]), conv[:V], conv[V:]

    def densify(self, scene: GaussianScene, adam, grad_accum, denom, normals, extent, grad_threshold=2e-4,
                percent_dense=0.01, min_opacity=0.005, capacity=None, stream=None):
        """Densification on deferred state (gs_densify): clone / split / prune
        of ``scene`` into a new GaussianScene (returned), from the accumulated
        view-space gradient norms ``grad_accum`` / ``denom`` (device fp32 [n])
        and standard-normal ``normals`` (device fp32 [2][3][n]) for the
        children of splits."""
        cap = int(capacity or 2 * scene.n)
        for _ in range(2):
            dst = GaussianScene(torch.zeros(scene.D, cap), scene.sh_degree, device=self.device,
                                with_rdir=scene.rdir_geo is not None, precision=scene.precision)
            sc, dc = scene.struct(), dst.struct()
            st = self.lib.gs_densify(self.h, C.byref(sc), C.byref(dc), C.byref(adam), _ptr(grad_accum.contiguous()),
                                     _ptr(denom.contiguous()), _ptr(normals.contiguous()), float(extent),
                                     float(grad_threshold), float(percent_dense), float(min_opacity), _stream(stream))
            if st == L.GS_ERR_CAPACITY and dc.n > cap:
                cap = int(dc.n)
                continue
            self._check(st, "gs_densify")
            dst.n, dst.step = int(dc.n), int(dc.step)
            return dst
        raise L.GsError(L.GS_ERR_CAPACITY, "gs_densify")

    def set_cull_wait_limit(self, first_wait):
        """Polls of each cull block's first wait on its own copies before it
        gives up and latches GS_ERR_TIMEOUT (default 2^24; failure-path tests)."""
        self._check(self.lib.gs_set_cull_wait_limit(self.h, int(first_wait)), "gs_set_cull_wait_limit")

    def set_raster_variant(self, v, bwd=None):
        """Pin the rasterizer variant (forward and backward, or ``bwd`` apart)."""
        if bwd is None:
            self._check(self.lib.gs_set_raster_variant(self.h, int(v)), "gs_set_raster_variant")
        else:
            self._check(self.lib.gs_set_raster_variants(self.h, int(v), int(bwd)), "gs_set_raster_variants")

    def timing_enable(self, max_steps):
        self._check(self.lib.gs_timing_enable(self.h, int(max_steps)), "gs_timing_enable")

    def timing_read(self, max_steps):
        """Per-step stage durations (ms) recorded with CUDA events inside gs_step:
        a list of dicts keyed by step, cull, fwd, bwd, adam, adam_apply."""
        buf = (C.c_float * (max_steps * len(L.SPANS)))()
        n = C.c_int32(0)
        self._check(self.lib.gs_timing_read(self.h, buf, int(max_steps), C.byref(n)), "gs_timing_read")
        k = len(L.SPANS)
        return [dict(zip(L.SPANS, buf[s * k:(s + 1) * k])) for s in range(n.value)]

    def raster_pair_counts(self, scene: GaussianScene, cam, stream=None):
        """(square-test pairs, contributing pairs, keys with no contributing pixel)
        of the backward for one view."""
        out = (C.c_uint64 * 3)()
        sc = scene.struct()
        cs = camera_struct(cam)
        self._check(self.lib.gs_raster_pair_counts(self.h, C.byref(sc), C.byref(cs), out, _stream(stream)),
                    "gs_raster_pair_counts")
        return int(out[0]), int(out[1]), int(out[2])

    def step_kernel_count(self):
        n = C.c_int32(0)
        self._check(self.lib.gs_step_kernel_count(self.h, C.byref(n)), "gs_step_kernel_count")
        return n.value

    def step(self, scene: GaussianScene, cams, targets, adam, loss=None, stream=None):
        nv = len(cams)
        cs = (L.Camera * nv)(*[camera_struct(c) for c in cams])
        tp = (C.c_void_p * nv)(*[t.data_ptr() for t in targets])
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        sc = scene.struct()
        st = self.lib.gs_step(self.h, C.byref(sc), cs, tp, nv, C.byref(adam), _ptr(loss), _stream(stream))
        self._check(st, "gs_step")
        scene.step = sc.step
        return loss


def _np_ptr(a, dtype):
    import numpy as np
    assert isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous, "contiguous numpy array expected"
    return a.ctypes.data


def cpu_deferred_step(w, m, v, plane0, uids, udelay, vids, grad, adam, step, threads=0):
    """Deferred optimizer step on host arrays (gs_cpu_deferred_step): w, m, v
    float32 [n][planes] numpy arrays, one row per Gaussian (updated in place),
    holding parameter rows plane0.. ; uids / udelay the update set; vids
    ascending ids with gradient rows grad float32 [len(vids)][planes]."""
    import numpy as np
    n_rows, planes = w.shape
    grow = grad.shape[1] if grad.ndim == 2 and grad.shape[1] else planes
    st = L.load().gs_cpu_deferred_step(_np_ptr(w, np.float32), _np_ptr(m, np.float32), _np_ptr(v, np.float32),
                                       n_rows, planes, int(plane0), planes, _np_ptr(uids, np.int32),
                                       _np_ptr(udelay, np.uint8), len(uids), _np_ptr(vids, np.int32),
                                       _np_ptr(grad, np.float32), len(vids), grow, C.byref(adam), int(step),
                                       int(threads))
    if st != L.GS_OK:
        raise L.GsError(st, "gs_cpu_deferred_step")


def cpu_forward(w, m, v, plane0, ids, counter, uids, udelay, vids, grad, adam, step, threads=0):
    """Parameter forwarding on host arrays (gs_cpu_forward): the values of
    Gaussians ``ids`` (with defer counters ``counter`` at step + 1) as step + 1
    sees them, float32 [planes][len(ids)] (w, m, v and grad as in
    cpu_deferred_step)."""
    import numpy as np
    n_rows, planes = w.shape
    n = len(ids)
    out = np.zeros((planes, max(n, 1)), np.float32)
    grow = grad.shape[1] if grad.ndim == 2 and grad.shape[1] else planes
    st = L.load().gs_cpu_forward(_np_ptr(w, np.float32), _np_ptr(m, np.float32), _np_ptr(v, np.float32), n_rows,
                                 planes, int(plane0), planes, _np_ptr(ids, np.int32), _np_ptr(counter, np.uint8), n,
                                 _np_ptr(uids, np.int32), _np_ptr(udelay, np.uint8), len(uids),
                                 _np_ptr(vids, np.int32), _np_ptr(grad, np.float32), len(vids), grow, C.byref(adam),
                                 int(step), _np_ptr(out, np.float32), out.shape[1], int(threads))
    if st != L.GS_OK:
        raise L.GsError(st, "gs_cpu_forward")
    return out[:, :n]


class _Render(torch.autograd.Function):
    """image = render(w) for a fixed visible set; the backward is gs_render_bwd
    followed by a scatter of the compact gradients to w's [D][pitch] layout."""

    @staticmethod
    def forward(fctx, w, gctx, scene, cam, ids, n_vis):
        img = gctx.render_fwd(scene, cam, ids, n_vis)
        fctx.gctx, fctx.scene, fctx.ids, fctx.n_vis = gctx, scene, ids, n_vis
        return img

    @staticmethod
    def backward(fctx, dimg):
        gc = fctx.gctx.render_bwd(dimg.contiguous(), fctx.scene.D)
        gfull = fctx.gctx.grad_scatter(fctx.scene, fctx.ids, fctx.n_vis, gc)
        return gfull, None, None, None, None, None


def render(gctx: Context, scene: GaussianScene, cam, ids, n_vis):
    """Differentiable render of one view with respect to ``scene.w``."""
    return _Render.apply(scene.w, gctx, scene, cam, ids, n_vis)


__all__ = ["Context", "GaussianScene", "render", "camera_struct", "adam_struct", "n_params", "cpu_deferred_step",
           "cpu_forward"]
