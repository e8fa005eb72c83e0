"""Benchmark of the 3DGS training hot path (GS-Scale, arXiv 2509.15645) on B300.

One step = one training iteration on one view: frustum cull of all Gaussians,
gather with deferred restore, tile rasterizer forward + L1 loss + backward,
deferred Adam (gs_step, replayed as a CUDA graph).  Workload: 10M Gaussians
on a 1x1 km aerial heightfield, SH degree 3, 1920x1080 nadir-to-oblique
views, FP32 (synthetic, seeded; see synth/scenes.py).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import re
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3DGS train steps/s at 10M Gaussians 1080p; cull+Adam HBM GB/s vs peak"
UNIT = "steps/s"
WORKLOAD = "aerial10m_1080p_sh3"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ---------------------------------------------------------------------------- replicas

def max_over_ranks(ms, dist, dev):
    """The slowest rank's time: the job ends when its last replica does.  With
    no process group (one GPU) the local time."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, ms):
    """Steps per second of the whole job: each of `world` replicas takes
    `steps` steps, and all of them finish within `ms` milliseconds."""
    return world * steps / (ms / 1e3)


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region: NVML
    (libnvidia-ml through ctypes) polled every ~2 ms from a thread, so a timed
    region of a few tens of ms still gets samples; else nvidia-smi every 100 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index, pci_bus_id=None):
        self.index, self.pci = index, pci_bus_id
        self.proc = self.thread = None
        self.samples = []
        self.nvml_error = None

    # clock event reason bits of the public NVML API (nvmlClocksEventReason*)
    REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def _nvml(self):
        """(sm_mhz(), reasons(), max_mhz) from libnvidia-ml through ctypes."""
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = C.c_void_p()
        if not (self.pci and lib.nvmlDeviceGetHandleByPciBusId_v2(self.pci.encode(), C.byref(h)) == 0):
            if lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.index), C.byref(h)) != 0:
                raise RuntimeError("no NVML handle")
        getr = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = C.c_uint(0)
        lib.nvmlDeviceGetMaxClockInfo(h, C.c_int(1), C.byref(mx))      # 1 = NVML_CLOCK_SM

        def sm_mhz():
            v = C.c_uint(0)
            return v.value if lib.nvmlDeviceGetClockInfo(h, C.c_int(1), C.byref(v)) == 0 else None

        def reasons():
            r = C.c_ulonglong(0)
            if getr(h, C.byref(r)) != 0:
                return []
            return [k for k, b in self.REASON_BITS.items() if r.value & b]

        return sm_mhz, reasons, mx.value

    def start(self):
        import threading
        try:
            sm_mhz, reasons, self.smax = self._nvml()
            self.stop_flag = threading.Event()

            def loop():
                while not self.stop_flag.is_set():
                    mhz = sm_mhz()
                    if mhz:
                        self.samples.append((mhz, reasons()))
                    time.sleep(0.002)

            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            return
        except Exception as e:
            self.thread = None
            self.nvml_error = repr(e)[:160]
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread:
            self.stop_flag.set()
            self.thread.join()
            sm = [x[0] for x in self.samples]
            reasons = sorted({r for x in self.samples for r in x[1]})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.smax, "reasons": reasons,
                    "samples": len(sm), "source": "nvml, ~2 ms"}
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(self.NAMES, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 100 ms",
                "nvml_error": self.nvml_error}


# ---------------------------------------------------------------------------- workload

def build_workload(n, n_views, seed_views=2, density_of=None, width=1920, height=1080):
    """The aerial workload; with density_of=N0 a scene of n Gaussians over the
    area that keeps the N0-Gaussian scene's density (same raster load per view)."""
    from synth import scenes
    scale, clusters = 5.0, 200
    if density_of:
        scale = 5.0 * math.sqrt(n / density_of)
        clusters = max(1, round(200 * n / density_of))
    cfg = scenes.cfg_aerial(n=n, n_views=n_views, seed_views=seed_views, scale=scale, n_clusters=clusters,
                            width=width, height=height)
    # the targets are images to fit: rendered from a seed-1 scene over the same
    # area, of at most 10M Gaussians (larger scenes would only lengthen the setup)
    nt = min(n, 10_000_000)
    tgt_scene = scenes.heightfield_scene(nt, seed=1, half_extent=cfg["half_extent"], amplitude=20.0,
                                         wavelength=(20.0 * scale, 25.0 * scale),
                                         n_clusters=max(1, round(clusters * nt / n)))
    return cfg, tgt_scene


def fp32_peak_tflops(sms, sm_max_mhz):
    """FP32 peak derived from unit counts and the clock: SMs (read from the
    device) x 128 FP32 lanes x 2 flops per FMA x the maximum SM clock."""
    return sms * 128 * 2 * sm_max_mhz * 1e6 / 1e12


# algorithmic FP32 operations of the rasterizer backward (one front-to-back
# pass) per (pixel, splat) pair: a contributing pair costs alpha (14), the
# transmittance and colour accumulation (8), the colour behind it and dL/dalpha
# (19), the colour gradients (6) and the conic / mean / opacity gradients (21);
# a pair inside the 3-sigma square that does not contribute costs alpha alone.
FLOPS_CONTRIB, FLOPS_SQUARE = 68.0, 14.0


def _int(x):
    """round() that maps a missing count (NaN) to None."""
    return None if x is None or not np.isfinite(x) else round(x)


def algorithmic_bytes(N, D, n_vis, n_upd, n_restore, bf16=False, n_cand=None):
    """Bytes the method must move per launch: the cull, the optimizer's apply
    sweep and its select pass (the minimum traffic of each, every byte read or
    written once)."""
    # cull: w of the mean and scale planes (0-5) for all, their restore
    # directions for Gaussians with a non-zero counter; the rotation planes
    # (6-9, w and direction) for the n_cand Gaussians that pass the
    # conservative pre-test; counters, bitmask, chunk counts
    if n_cand is None:
        n_cand = N
    restore_frac = n_restore / max(N, 1)
    cull = (24.0 * N + 24.0 * n_restore + n_cand * (16.0 + 16.0 * restore_frac)
            + 1.0 * N + N / 8.0 + 4.0 * N / 2048.0)
    # apply: w, m, v read + w, m, v written per parameter of each update-set
    # member, and the restore direction of each geometry plane written;
    # gradients of the visible ones, ids and delays.  bf16 forms: the 11
    # geometry planes keep fp32 w and direction with bf16 m, v (20 B); SH
    # planes hold bf16 w, m, v (12 B)
    per_member = (20.0 * 11 + 12.0 * (D - 11)) if bf16 else 28.0 * 11 + 24.0 * (D - 11)
    apply = per_member * n_upd + 4.0 * D * n_vis + 4.0 * n_upd + 1.0 * n_upd
    select = 2.0 * N + N / 4.0
    return cull, apply, select


def method_bytes(N, D, n_vis, n_upd, bf16=False):
    """The method's algorithmic bytes per step for the cull and the deferred
    update, as planned from the paper's algorithm (restore reading w, m and v;
    every Gaussian's geometry planes read once): cull 121 N + N/8 + 4 |V| in
    fp32 (w, m, v of the 10 geometry planes and the counter), 81 N + ... with
    bf16 moments; update 2 N (counters) + 28 D |U| (w, m, v read and written)
    + 4 |V| in fp32, 2 N + (11 * 20 + (D - 11) * 16) |U| + 4 |V| with bf16 SH
    and moments.  The kernels move less (restore directions instead of m and v,
    rotation planes only for the pre-test's survivors): `algorithmic_bytes`."""
    cull = (81.0 if bf16 else 121.0) * N + N / 8.0 + 4.0 * n_vis
    per_member = (11 * 20.0 + (D - 11) * 16.0) if bf16 else 28.0 * D
    adam = 2.0 * N + per_member * n_upd + 4.0 * n_vis
    return cull, adam


def run_ours(args):
    import torch
    import paper_2509_15645_b300 as gs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    N = args.gaussians
    IW, IH = (int(x) for x in args.image.split("x"))
    vps = args.views_per_step
    cfg, tgt_params = build_workload(N, args.views, seed_views=2 + rank, density_of=args.density_of, width=IW,
                                     height=IH)
    cams = cfg["cams"]
    deg = cfg["sh_degree"]
    D = 11 + 3 * (deg + 1) ** 2
    H, W = cams[0].height, cams[0].width

    tile = tuple(int(x) for x in args.tile.split("x"))
    # capacities: visible set and keys per view scale with the image area (a
    # 10M-density aerial view of 1920x1080 sees ~0.65M Gaussians, ~3.4M keys)
    area = W * H / (1920 * 1080)
    max_vis = int(min(N, max(0.6 * N if not args.density_of else 0, 3_000_000 * area * (args.density_of or N) / 10e6)))
    max_vis = int(min(N, max(max_vis, 1_000_000)))
    max_keys = int(min(160_000_000, max(16_000_000, 20 * max_vis)))
    # list-order records (48 B per key of capacity) let the autotuner weigh the
    # TMA-staged rasterizer variant; not under an HBM budget
    ctx_kw = dict(max_gaussians=N, max_visible=max_vis, max_keys=max_keys, max_width=W, max_height=H, tile=tile,
                  max_views=vps, max_sh_degree=deg, list_records=0 if args.budget_gb else 1)
    # HBM budget: state that does not fit goes to the host tier (SH planes and
    # their optimizer state in pinned host memory, streamed by gs_step)
    tier, stage_chunks, plan, eb = gs.GS_TIER_DEVICE, 0, None, 4
    if args.cpu_optimizer:
        # the paper's offloaded configuration: SH planes and their moments in
        # host memory, stepped by the host cores (parameter forwarding, deferred update)
        tier = gs.GS_TIER_HOST_CPU_OPT
        args.no_bf16, args.bf16_only = True, False
        plan = {"tier": "host_cpu_optimizer", "device_state_gb": round(N * (44 + 2 * 11 * 4 + 44 + 1) / 1e9, 2),
                "host_state_gb": round(N * (D - 11) * 12 / 1e9, 2)}
    elif args.budget_gb:
        prec0 = gs.GS_BF16_SH_MOM if args.bf16_only else gs.GS_FP32
        eb = 4 if prec0 == gs.GS_FP32 else 2
        resident = N * (44 + (D - 11) * eb + 2 * D * eb + 44 + (D - 11) * eb + 1)
        geo_only = N * (44 + 2 * 11 * eb + 44 + 1)
        ws0 = gs.Context.workspace_bytes(**ctx_kw)
        budget = args.budget_gb * 1e9
        if resident + ws0 > budget:
            R = 1 << args.chunk_shift
            ring_chunk = 3 * (D - 11) * R * eb          # w, m, v rows of the SH type
            stage_chunks = int((budget - geo_only - ws0) // ring_chunk)
            if stage_chunks < 1:
                raise SystemExit(f"budget {args.budget_gb} GB holds no staging ring")
            tier = gs.GS_TIER_HOST_SH
        plan = {"budget_gb": args.budget_gb, "resident_state_gb": round(resident / 1e9, 2),
                "workspace_gb": round(ws0 / 1e9, 2),
                "tier": "host_sh" if tier == gs.GS_TIER_HOST_SH else "device",
                "device_state_gb": round((geo_only if tier else resident) / 1e9, 2),
                "stage_chunks": stage_chunks, "chunk_rows": 1 << args.chunk_shift}
    ctx = gs.Context(**ctx_kw, device=local, stage_chunks=stage_chunks, chunk_shift=args.chunk_shift,
                     stage_elem_bytes=eb if stage_chunks else 0, cpu_opt=1 if args.cpu_optimizer else 0)
    if args.cpu_threads:
        ctx.set_cpu_threads(args.cpu_threads)

    def finish():
        """The last step's host-side work: the host tier's write-backs, or the
        held SH update of the host-core optimizer."""
        if tier == gs.GS_TIER_HOST_CPU_OPT:
            ctx.sync_status()
        else:
            ctx.wait_copies()
    # targets: the seed-1 scene rendered by the same library (setup, untimed)
    tscene = gs.GaussianScene(tgt_params, deg, device=dev, with_optimizer=False)
    del tgt_params
    targets = []
    for cam in cams:
        ids, nv = ctx.cull(tscene, cam)
        targets.append(ctx.render_fwd(tscene, cam, ids, nv).clone())
    ctx.sync_status()
    del tscene
    P0 = cfg.pop("scene")
    torch.cuda.empty_cache()
    adam = gs.adam_struct(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-15, max_defer=15, seed=1)
    loss = torch.zeros(1, device=dev)
    stream = torch.cuda.current_stream()
    K, Wm = args.steps, args.warmup
    tcap = max(Wm + K, 16) + 8
    peak, peak_src = _peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sms = props.multi_processor_count
    try:
        sm_max = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except Exception:
        sm_max = 2032.0
    fp32_peak = fp32_peak_tflops(n_sms, sm_max)
    pci = getattr(props, "pci_bus_id", None)
    pci = f"{getattr(props, 'pci_domain_id', 0):08x}:{pci:02x}:{getattr(props, 'pci_device_id', 0):02x}.0" \
        if isinstance(pci, int) else None
    gbs = lambda b, ms: b / (ms * 1e-3) / 1e9 if ms else None

    def one_step(sc, s, tgt=None):
        vs = [(s * vps + j) % len(cams) for j in range(vps)]
        ctx.step(sc, [cams[v] for v in vs], tgt or [targets[v] for v in vs], adam, loss=loss)

    def link_rates(nbytes=1 << 30, reps=4):
        """Host<->device copy rates of this GPU's link from pinned memory (GB/s):
        H2D alone, D2H alone, and both directions at once (their sum), untimed
        setup measurements for the host tier."""
        h = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in range(2)]
        d = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]
        st = [torch.cuda.Stream(device=dev) for _ in range(2)]

        def run(up, down):
            torch.cuda.synchronize()
            t = time.perf_counter()
            for _ in range(reps):
                if up:
                    with torch.cuda.stream(st[0]):
                        d[0].copy_(h[0], non_blocking=True)
                if down:
                    with torch.cuda.stream(st[1]):
                        h[1].copy_(d[1], non_blocking=True)
            torch.cuda.synchronize()
            return round(reps * nbytes * (up + down) / (time.perf_counter() - t) / 1e9, 1)

        run(1, 1)
        out = {"h2d": run(1, 0), "d2h": run(0, 1), "both_directions": run(1, 1)}
        del h, d
        return out

    def trace_step(sc, s):
        """One extra untimed step under the CUDA activity trace: the kernels of
        this library it launches (for steps that run without a captured graph,
        e.g. the host tier) and, per copy direction, the bytes, the summed copy
        durations and the span from the first copy's start to the last's end."""
        try:
            import tempfile
            from torch.profiler import profile, ProfilerActivity
            torch.cuda.synchronize()
            with profile(activities=[ProfilerActivity.CUDA]) as prof:
                one_step(sc, s)
                torch.cuda.synchronize()
            with tempfile.NamedTemporaryFile(suffix=".json") as f:
                prof.export_chrome_trace(f.name)
                ev = json.load(open(f.name)).get("traceEvents", [])
            kernels = sum(1 for e in ev if e.get("cat") == "kernel" and re.search(r"(^|[\s:])k_\w+", e.get("name", "")))
            copies = {}
            for d, key in (("HtoD", "h2d"), ("DtoH", "d2h")):
                cs = [e for e in ev if e.get("cat") == "gpu_memcpy" and d in e.get("name", "")]
                if cs:
                    nb = sum(float(e.get("args", {}).get("bytes", 0)) for e in cs)
                    busy = sum(float(e["dur"]) for e in cs) * 1e-3
                    span = (max(e["ts"] + e["dur"] for e in cs) - min(e["ts"] for e in cs)) * 1e-3
                    copies[key] = {"copies": len(cs), "bytes": nb, "busy_ms": round(busy, 3),
                                   "span_ms": round(span, 3), "gbs_while_busy": round(nb / busy * 1e-6, 1)}
            return kernels, copies
        except Exception as e:
            return None, {"error": repr(e)[:200]}

    def timed_steps(sc):
        """W warm-up steps, then K steps between CUDA events on the launching
        stream (barrier + synchronize on both sides), clocks sampled meanwhile.
        Returns (ms over the K steps, max over ranks; per-step stage spans; clocks)."""
        ctx.timing_enable(tcap)
        for s in range(Wm):
            one_step(sc, s)
        ctx.sync_status()
        ctx.timing_read(tcap)            # discard warm-up timings
        clocks = ClockSampler(local, pci)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        staged = []
        for s in range(K):
            one_step(sc, Wm + s)
            if tier == gs.GS_TIER_HOST_SH:     # host-side counters of the step just enqueued (no synchronisation)
                staged.append(ctx.host_tier_stats())
            elif tier:
                staged.append(ctx.cpu_tier_stats())
        finish()                         # the last step's write-backs / held update are timed too
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clk = clocks.stop()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        sp = ctx.timing_read(tcap)
        ctx.sync_status()
        ms = max_over_ranks(ms, dist, dev)
        return ms, sp, clk, staged

    def measure(precision):
        """Autotune, time K steps of one precision form, then an untimed pass
        over the views for the counts behind the algorithmic bytes and flops."""
        sc = gs.GaussianScene(P0, deg, device=dev, precision=precision, tier=tier)
        if tier == gs.GS_TIER_DEVICE and args.raster_variant is None:
            variant, ms_f, ms_b = ctx.autotune(sc, cams[0])     # rasterizer variants for this workload (untimed)
            variant_ms = {"fwd_stage": ms_f, "bwd_stage": ms_b}
        elif tier == gs.GS_TIER_DEVICE:
            variant, variant_ms = None, {}                       # pinned below
        else:   # the autotuner renders through the resident path: the warp tiles it picks on the resident 10M step
            variant, variant_ms = (7, 7), {}
            ctx.set_raster_variant(7, 7)
        if args.raster_variant is not None:
            fb = [int(x) for x in str(args.raster_variant).split(",")]
            variant = (fb[0], fb[-1])
            ctx.set_raster_variant(variant[0], variant[1])
        ms_total, spans, clk, staged = timed_steps(sc)
        stats = []
        ctx.timing_enable(tcap)
        for s in range(min(len(cams), 16 if tier == gs.GS_TIER_DEVICE else 4)):
            n_restore_geo = int((sc.counter[:N] > 0).sum().item())
            one_step(sc, Wm + K + s)
            c = ctx.counters().cpu().tolist()
            stats.append((c[0], c[1], c[2], n_restore_geo, c[6], c[7]))
        ctx.timing_read(tcap)
        kernels = ctx.step_kernel_count()    # kernel nodes of the captured step graph
        copy_trace = None
        if not kernels:
            kernels, copy_trace = trace_step(sc, Wm + K + 16)
        if tier == gs.GS_TIER_DEVICE:
            pairs = np.array([ctx.raster_pair_counts(sc, cam) for cam in cams], np.float64)   # untimed
        else:
            pairs = np.full((1, 3), np.nan)
        st = {}
        for k in ("step", "cull", "fwd", "bwd", "adam", "adam_apply", "raster_bwd"):
            vals = [x[k] for x in spans if x[k] >= 0]
            st[k] = float(np.mean(vals)) if vals else None
        m = {"sc": sc, "ms": ms_total, "clk": clk, "st": st, "variant": variant, "variant_ms": variant_ms,
             "n_vis": float(np.mean([x[0] for x in stats])), "n_keys": float(np.mean([x[1] for x in stats])),
             "n_upd": float(np.mean([x[2] for x in stats])), "n_rest": float(np.mean([x[3] for x in stats])),
             "n_fp64": float(np.mean([x[4] for x in stats])), "n_cand": float(np.mean([x[5] for x in stats])),
             "sq_pairs": float(pairs[:, 0].mean()), "on_pairs": float(pairs[:, 1].mean()),
             "empty_keys": float(pairs[:, 2].mean()),
             "kernels": kernels, "copy_trace": copy_trace,
             "staged_chunks": (float(np.mean([x[0] for x in staged]))
                               if staged and tier == gs.GS_TIER_HOST_SH else None),
             "staged_bytes": (float(np.mean([x[1] for x in staged]))
                              if staged and tier == gs.GS_TIER_HOST_SH else None),
             "cpu_stats": ({k: float(np.mean([x[k] for x in staged])) for k in staged[0]}
                           if staged and tier == gs.GS_TIER_HOST_CPU_OPT else None)}
        b_cull, b_apply, b_select = algorithmic_bytes(N, D, m["n_vis"], m["n_upd"], m["n_rest"],
                                                      bf16=precision != gs.GS_FP32, n_cand=m["n_cand"])
        m.update(b_cull=b_cull, b_apply=b_apply, b_select=b_select)
        m["cull_adam"] = {
            "cull_gbs": gbs(b_cull, st["cull"]), "adam_apply_gbs": gbs(b_apply, st["adam_apply"]),
            "adam_stage_gbs": gbs(b_apply + b_select, st["adam"]),
            "cull_plus_adam_gbs": gbs(b_cull + b_apply + b_select, (st["cull"] or 0) + (st["adam"] or 0)),
            "peak_gbs": peak, "cull_bytes": round(b_cull), "adam_bytes": round(b_apply + b_select)}
        ca = m["cull_adam"]
        ca["cull_plus_adam_frac"] = ca["cull_plus_adam_gbs"] and ca["cull_plus_adam_gbs"] / peak
        mb_cull, mb_adam = method_bytes(N, D, m["n_vis"], m["n_upd"], bf16=precision != gs.GS_FP32)
        ca["method_bytes"] = round(mb_cull + mb_adam)
        ca["cull_plus_adam_method_gbs"] = gbs(mb_cull + mb_adam, (st["cull"] or 0) + (st["adam"] or 0))
        ca["cull_plus_adam_method_frac"] = ca["cull_plus_adam_method_gbs"] and ca["cull_plus_adam_method_gbs"] / peak
        for k in list(ca):
            if isinstance(ca[k], float):
                ca[k] = round(ca[k], 4 if k.endswith("frac") else 1)
        return m

    # DRAM bytes per launch of the rasterizer backward on this workload (10M,
    # 1920x1080, one view), by variant, from ncu captures of
    # dram__bytes_read.sum + dram__bytes_write.sum of the kernels as they are
    # (profiles/launches_aerial10m_1080p.md); variants 8 and 9 changed since
    # their captures (None); other workloads: not captured
    RASTER_BWD_TRAFFIC = {7: 127.9e6, 8: None, 9: None}

    def roofline(m):
        """Roofline entry of the kernel with the largest live event time per step."""
        st = m["st"]
        flops = FLOPS_CONTRIB * m["on_pairs"] + FLOPS_SQUARE * (m["sq_pairs"] - m["on_pairs"])
        cands = {"k_raster_bwd": st["raster_bwd"] or 0.0, "k_adam_apply": st["adam_apply"] or 0.0,
                 "k_cull": st["cull"] or 0.0}
        if not np.isfinite(flops):
            cands.pop("k_raster_bwd")      # no pair counts (host tier)
        dom = max(cands, key=cands.get)
        if dom == "k_raster_bwd":
            ach = flops / (st["raster_bwd"] * 1e-3) / 1e12
            return {"kernel": dom, "bound": "alu", "achieved": round(ach, 3), "peak": round(fp32_peak, 2),
                    "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4),
                    "peak_source": f"derived: {n_sms} SMs (device attribute) x 128 FP32 lanes x 2 flop/FMA x "
                                   f"{sm_max:g} MHz (maximum SM clock)",
                    "algorithmic_flops_per_launch": round(flops),
                    "traffic": (RASTER_BWD_TRAFFIC.get(m["variant"][1]) if cfg_note == WORKLOAD and m["variant"]
                                else None),
                    "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"}
        b = m["b_apply"] if dom == "k_adam_apply" else m["b_cull"]
        t = st["adam_apply"] if dom == "k_adam_apply" else st["cull"]
        return {"kernel": dom, "bound": "hbm", "achieved": round(gbs(b, t), 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs(b, t) / peak, 4), "peak_source": peak_src,
                "algorithmic_bytes_per_launch": round(b), "traffic": None}

    def e2e(sc):
        """Steps/s through the public API with the step's targets copied from
        pinned host memory and the loss read back, every step.  The targets are
        double-buffered: step s + 1's copy runs on a copy stream while step s
        computes (events order each buffer's copy before its use and its reuse
        after the step that read it), as a data loader would feed training."""
        host_t = [t.cpu().pin_memory() for t in targets]
        bufs = [[torch.empty_like(targets[0]) for _ in range(vps)] for _ in range(2)]
        host_loss = torch.zeros(1).pin_memory()
        cstream = torch.cuda.Stream(device=dev)
        copied = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        for e in used:
            e.record(stream)

        def prefetch(s):
            b = s % 2
            with torch.cuda.stream(cstream):
                cstream.wait_event(used[b])              # the step that read this buffer is done
                for j in range(vps):
                    bufs[b][j].copy_(host_t[(s * vps + j) % len(cams)], non_blocking=True)
                copied[b].record(cstream)

        def e2e_step(s, last):
            b = s % 2
            stream.wait_event(copied[b])
            one_step(sc, s, tgt=bufs[b])
            used[b].record(stream)
            host_loss.copy_(loss, non_blocking=True)
            if not last:
                prefetch(s + 1)

        ctx.timing_enable(0)
        prefetch(0)
        for s in range(max(Wm, 3)):
            e2e_step(s, False)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        cstream.wait_stream(stream)      # the timed region's first copy starts after f0
        prefetch(0)
        for s in range(K):
            e2e_step(s, s == K - 1)
        finish()
        f1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(f0.elapsed_time(f1), dist, dev)
        ctx.sync_status()
        return {"value": round(job_rate(world, K, ms), 4), "unit": UNIT,
                "h2d_bytes_per_step": int(targets[0].numel() * 4 * vps), "d2h_bytes_per_step": 4,
                "copies": "targets double-buffered on a copy stream (step s+1's copy overlaps step s)"}

    if args.density_of or (IW, IH) != (1920, 1080) or vps != 1:
        cfg_note = f"aerial{N / 1e6:g}m" + (f"_at_density_of_{args.density_of / 1e6:g}m" if args.density_of else "") + \
            f"_{IW}x{IH}_sh3" + (f"_{vps}views" if vps > 1 else "")
    else:
        cfg_note = WORKLOAD
    main_prec = gs.GS_BF16_SH_MOM if args.bf16_only else gs.GS_FP32
    if args.budget_gb:
        args.no_bf16 = True        # the memory plan was made for one form
    m = measure(main_prec)
    e2e_main = e2e(m["sc"])
    bf16 = None
    if not args.bf16_only and not args.no_bf16:
        # the precision form: bf16 SH coefficients and moments, fp32 geometry
        # (same initial parameters, views and targets; its own warm-up and timed steps)
        del m["sc"]
        torch.cuda.empty_cache()
        mb = measure(gs.GS_BF16_SH_MOM)
        del mb["sc"]
        bf16 = {"form": "bf16_sh_mom (bf16 SH and moments, stochastic rounding; fp32 geometry and compositing)",
                "value": round(job_rate(world, K, mb["ms"]), 4), "unit": UNIT, "ms_per_step": round(mb["ms"] / K, 4),
                "stages_ms": {k: (round(v, 4) if v is not None else None) for k, v in mb["st"].items()},
                "cull_adam": mb["cull_adam"], "roofline": roofline(mb), "clocks": mb["clk"],
                "update_set": round(mb["n_upd"]), "state_bytes_per_gaussian": 11 * 4 * 2 + (D - 11) * 2 + D * 2 * 2 + 1}
    K_ms = m["ms"]
    out = {
        "metric": METRIC, "value": round(job_rate(world, K, K_ms), 4), "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": round(K_ms / K, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded aerial heightfield, random-init Gaussians)",
        "config": {"workload": cfg_note, "gaussians": N, "image": f"{W}x{H}", "sh_degree": deg,
                   "views_per_step": vps, "memory_plan": plan, "form": "bf16_sh_mom" if args.bf16_only else "plain_fp32",
                   "adam": "deferred", "tile": args.tile,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": f"inputs larger than L2 (parameters + moments {N * D * 12 / 1e9:.1f} GB in fp32), no flush",
                   "visible_per_view": round(m["n_vis"]), "keys_per_view": round(m["n_keys"]),
                   "update_set": round(m["n_upd"]), "fp64_covariances_per_view": round(m["n_fp64"]),
                   "cull_pretest_survivors": round(m["n_cand"]),
                   "square_pairs_per_view": _int(m["sq_pairs"]), "contrib_pairs_per_view": _int(m["on_pairs"]),
                   "keys_without_contributor_per_view": _int(m["empty_keys"]),
                   "raster_variant": {"fwd": m["variant"][0], "bwd": m["variant"][1]},
                   "autotune_ms": {k: [None if t is None else round(t, 4) for t in v]
                                   for k, v in m["variant_ms"].items()}},
        "roofline": roofline(m),
        "cull_adam": m["cull_adam"],
        "stages_ms": {k: (round(v, 4) if v is not None else None) for k, v in m["st"].items()},
        "e2e": e2e_main,
        "clocks": m["clk"],
        "gpu_launches": int(m["kernels"] * K) if m["kernels"] else None,
        "bf16_form": bf16,
    }
    if tier == gs.GS_TIER_HOST_CPU_OPT:
        cs = m["cpu_stats"]
        out["cpu_optimizer"] = {
            "threads": args.cpu_threads or os.cpu_count(),
            "forward_ms_per_step": round(cs["forward_ms"], 3), "host_update_ms_per_step": round(cs["update_ms"], 3),
            "wait_for_update_ms_per_step": round(cs["wait_ms"], 3),
            "h2d_bytes_per_step": round(cs["h2d_bytes"]), "d2h_bytes_per_step": round(cs["d2h_bytes"]),
            "rows_forwarded_per_step": round(cs["rows"]), "update_set_per_step": round(cs["held_members"]),
            "copy_trace": m["copy_trace"]}
        out["roofline"] = {"bound": "host", "note": "host-core optimizer: the step is bound by the host's "
                           "forwarding and deferred update; kernel rooflines are measured on the resident workloads"}
        out["cull_adam"] = None
    elif tier:
        out["host_tier"] = {"staged_chunks_per_step": m["staged_chunks"], "chunk_rows": 1 << args.chunk_shift,
                            "bytes_per_step": m["staged_bytes"],
                            "pcie_gbs": m["staged_bytes"] / (K_ms / K * 1e-3) / 1e9 if m["staged_bytes"] else None,
                            "copy_trace": m["copy_trace"], "link_gbs": link_rates()}
        # the counts behind the kernels' algorithmic bytes come from untimed steps at
        # another point of the deferral cycle than the timed ones: no kernel roofline here
        out["roofline"] = {"bound": "pcie", "note": "host tier: the step is bound by its host<->device copies; "
                           "kernel rooflines are measured on the resident workloads"}
        out["cull_adam"] = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, sample_frac=0.1)
    if rank == 0 and world == 1 and args.extra_forms and not (args.bf16_only or args.budget_gb or vps != 1 or
                                                               args.density_of):
        out.update(extra_forms(args))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def extra_forms(args):
    """The batched BF16 form, the host-offload configuration and the paper's
    host-core optimizer configuration, each timed by this script in a
    subprocess of its own (same K and W) after the main line:
    batched_bf16 = 10M resident, 4 views of 1600x1200 per step, bf16 SH and
    moments; host_tier_40m = 40M Gaussians on the 2x2 km field (the 10M
    field's density) with a 24 GB
    HBM budget (SH planes and their moments in pinned host memory), 4 views of
    1600x1200 per step, fp32 and bf16; cpu_optimizer_40m = the same 40M
    workload in the paper's own offloaded configuration (SH planes and their
    moments in host memory, stepped by the host cores: parameter forwarding
    and the deferred update, §4.2.2 and §4.3), fp32."""
    runs = {"batched_bf16": ["--bf16-only", "--views-per-step", "4", "--image", "1600x1200"],
            "host_tier_40m_fp32": ["--gaussians", "40000000", "--density-of", "10000000", "--budget-gb", "24",
                                   "--views-per-step", "4", "--image", "1600x1200"],
            "host_tier_40m_bf16": ["--gaussians", "40000000", "--density-of", "10000000", "--budget-gb", "24",
                                   "--views-per-step", "4", "--image", "1600x1200", "--bf16-only"],
            "cpu_optimizer_40m": ["--gaussians", "40000000", "--density-of", "10000000", "--cpu-optimizer",
                                  "--views-per-step", "4", "--image", "1600x1200"]}
    out = {}
    for name, extra in runs.items():
        cmd = [sys.executable, os.path.abspath(__file__), "--steps", str(args.steps), "--warmup", str(args.warmup),
               "--no-cpu-baseline", "--no-extra-forms", *extra]
        t0 = time.time()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
            line = [x for x in r.stdout.strip().splitlines() if x.startswith("{")]
            sub = json.loads(line[-1]) if r.returncode == 0 and line else {"error": (r.stderr or r.stdout)[-400:]}
        except Exception as e:
            sub = {"error": repr(e)[:400]}
        keep = ("value", "unit", "ms_per_step", "stages_ms", "cull_adam", "roofline", "clocks", "e2e", "config",
                "host_tier", "cpu_optimizer", "gpu_launches", "error")
        out[name] = {k: sub[k] for k in keep if k in sub}
        out[name]["wall_s"] = round(time.time() - t0, 1)
    return out


# ---------------------------------------------------------------------------- image splitting (§4.4)

def run_config_timings(args):
    """The GPU path on the smaller workload definitions (after autotuning,
    CUDA events over K steps after W warm-ups): the 10k-Gaussian 64x64 step
    (gs_step, SH 0, 16x16 tiles); the 1M heightfield's 1080p orbit (gs_step over
    the orbit's views in turn, deferred Adam, 8x4 tiles); the 200k 512x512
    differentiation case (gs_render_fwd + gs_render_bwd through the C ABI,
    16x16 tiles).  Inputs resident, no flush (these are small)."""
    import torch
    import paper_2509_15645_b300 as gs
    from synth import scenes
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    K, Wm = args.steps, max(args.warmup, 3)
    stream = torch.cuda.current_stream()
    out = {"metric": "GPU ms per step on the small workload definitions", "unit": "ms", "steps": K, "warmup": Wm,
           "results": {}}

    def timed(fn):
        for s in range(Wm):
            fn(s)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(K):
            fn(Wm + s)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    def step_case(c, tile, views):
        P, deg = c["scene"], c["sh_degree"]
        n = P.shape[1]
        cams = c["cams"][:views]
        W, H = cams[0].width, cams[0].height
        ctx = gs.Context(max_gaussians=n, max_visible=n, max_keys=min(64 * n, 80_000_000), max_width=W,
                         max_height=H, tile=tile, max_sh_degree=deg)
        ts = gs.GaussianScene(c["target_scene"], deg, with_optimizer=False)
        tg = []
        for cam in cams:
            ids, nv = ctx.cull(ts, cam)
            tg.append(ctx.render_fwd(ts, cam, ids, nv).clone())
        del ts
        sc = gs.GaussianScene(P, deg)
        ctx.autotune(sc, cams[0])
        adam = gs.adam_struct(lr=1e-3, eps=1e-15)
        loss = torch.zeros(1, device=dev)
        ms = timed(lambda s: ctx.step(sc, [cams[s % len(cams)]], [tg[s % len(cams)]], adam, loss=loss))
        ctx.sync_status()
        return round(ms, 4), int(ctx.counters()[0].item())

    c1 = scenes.cfg_small_step()
    ms, nv = step_case(c1, (16, 16), 1)
    out["results"]["cube10k_64px_sh0_step"] = {"ms": ms, "steps_per_s": round(1e3 / ms, 1), "visible": nv}
    c2 = scenes.cfg_heightfield_1m()
    ms, nv = step_case(c2, (8, 4), 100)
    out["results"]["heightfield1m_1080p_orbit_step"] = {"ms": ms, "steps_per_s": round(1e3 / ms, 1),
                                                         "visible_last_view": nv}
    c3 = scenes.cfg_diff_check()
    P, deg, cam = c3["scene"], c3["sh_degree"], c3["cams"][0]
    n = P.shape[1]
    ctx = gs.Context(max_gaussians=n, max_visible=n, max_keys=20_000_000, max_width=cam.width, max_height=cam.height,
                     tile=(16, 16), max_sh_degree=deg)
    sc = gs.GaussianScene(P, deg, with_optimizer=False)
    ids, nv = ctx.cull(sc, cam)
    dimg = torch.randn(3, cam.height, cam.width, device=dev)

    def fwd_bwd(s):
        ctx.render_fwd(sc, cam, ids, nv)
        ctx.render_bwd(dimg, sc.D)

    ms = timed(fwd_bwd)
    ctx.sync_status()
    out["results"]["cube200k_512px_sh3_fwd_bwd"] = {"ms": round(ms, 4), "visible": int(nv.item())}
    print(json.dumps(out), flush=True)


def run_split_demo(args):
    """Balance-aware image splitting (§4.4) on a view that crosses mem_limit:
    1M Gaussians on the 200 x 200 m heightfield, one 1920x1080 view from 100 m
    altitude, 80 m off-centre, looking at the origin (about 42% of the
    Gaussians visible).  Three contexts, each sized to the counts it must hold
    (measured first, +10%): the view whole; its two regions (gs_split_point,
    5 rounds) rendered one after the other through one set of render buffers
    (render_views = 1); the two regions rendered together (render_views = 2).
    Reports each one's workspace, the peak device memory of its steps (torch's
    allocator: scene state + workspace + targets), and its step time (CUDA
    events over --steps steps of the same view)."""
    import torch
    import paper_2509_15645_b300 as gs
    from synth import scenes
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n, deg, W, H = 1_000_000, 3, 1920, 1080
    P = scenes.heightfield_scene(n, seed=0)
    T = scenes.heightfield_scene(n, seed=1)
    cam = scenes.camera_lookat((80.0, 0.0, 100.0), (0.0, 0.0, 0.0), W, H, 60.0)
    adam = gs.adam_struct(lr=1e-3, eps=1e-15)
    big = dict(max_gaussians=n, max_visible=n, max_keys=60_000_000, max_width=W, max_height=H, tile=(8, 4),
               max_sh_degree=deg)
    # target and the counts that size the contexts
    probe = gs.Context(**big, max_views=2)
    ts = gs.GaussianScene(T, deg, with_optimizer=False)
    ids, nv = probe.cull(ts, cam)
    target = probe.render_fwd(ts, cam, ids, nv).clone()
    del ts
    sc = gs.GaussianScene(P, deg)
    frac = None
    ids, nv = probe.cull(sc, cam)
    probe.render_fwd(sc, cam, ids, nv)
    probe.sync_status()
    n_vis, n_keys = int(nv.item()), int(probe.counters()[1].item())
    frac = n_vis / n
    regions = probe.plan_split(sc, cam, adam, mem_limit=0.3)
    assert regions is not None, "the view does not cross mem_limit"
    reg_counts = []
    for r in regions:
        ids, nv = probe.cull(sc, r)
        probe.render_fwd(sc, r, ids, nv)
        probe.sync_status()
        reg_counts.append((int(nv.item()), int(probe.counters()[1].item())))
    del probe
    torch.cuda.empty_cache()
    res = {}
    for name, views, rv, vis, keys in (
            ("whole_view", 1, 0, n_vis, n_keys),
            ("split_sequential", 2, 1, max(c[0] for c in reg_counts), max(c[1] for c in reg_counts)),
            ("split_together", 2, 2, max(c[0] for c in reg_counts), max(c[1] for c in reg_counts))):
        kw = dict(big, max_visible=int(vis * 1.1) + 1024, max_keys=int(keys * 1.1) + 4096)
        ws = gs.Context.workspace_bytes(**kw, max_views=views, render_views=rv)
        sc = gs.GaussianScene(P, deg)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        ctx = gs.Context(**kw, max_views=views, render_views=rv)
        cams = [cam] if views == 1 else regions
        tg = [target] if views == 1 else [r.crop(target) for r in regions]
        loss = torch.zeros(1, device=dev)
        for _ in range(args.warmup):
            ctx.step(sc, cams, tg, adam, loss=loss)
        ctx.sync_status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            ctx.step(sc, cams, tg, adam, loss=loss)
        e1.record()
        torch.cuda.synchronize()
        ctx.sync_status()
        res[name] = {"workspace_gb": round(ws / 1e9, 3), "peak_device_gb": round(torch.cuda.max_memory_allocated() / 1e9, 3),
                     "ms_per_step": round(e0.elapsed_time(e1) / args.steps, 4), "capacity_visible": kw["max_visible"],
                     "capacity_keys": kw["max_keys"], "loss": round(loss.item(), 6)}
        del ctx, sc
        torch.cuda.empty_cache()
    out = {"metric": "image splitting: peak device memory and step time, split vs whole view", "unit": "GB, ms",
           "workload": "heightfield1m_1080p_sh3, view from 100 m altitude, 80 m off-centre", "gaussians": n,
           "visible_fraction": round(frac, 4), "mem_limit": 0.3,
           "split": {"axis": "x" if regions[0].height == H else "y",
                     "at_px": regions[1].x0 if regions[0].height == H else regions[1].y0,
                     "regions_visible_keys": reg_counts},
           "results": res, "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic"}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------- oracle (CPU)

def _oracle_step(orc, P, deg, cam, target, W_, M_, V_, C_, t, hp):
    r = orc.render_loss_backward(P if W_ is None else W_, deg, cam, target)
    kept = np.nonzero(r["splats"]["keep"])[0].astype(np.int32)
    orc.adam_deferred(W_, M_, V_, C_, kept, r["grad"][:, kept], t, hp)
    return r["loss"], kept.size


def oracle_sample(frac, seed=0):
    """A random `frac` of the workload's Gaussians (oracle baseline sample)."""
    from synth import scenes
    cfg = scenes.cfg_aerial(n=10_000_000, n_views=16, seed_views=2)
    P = cfg["scene"]
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(P.shape[1], int(P.shape[1] * frac), replace=False))
    Ps = np.ascontiguousarray(P[:, sel]).astype(np.float64)
    del P, cfg["scene"]
    return Ps, cfg


def cpu_baseline(args, sample_frac=0.1, steps=1):
    from oracle import oracle as orc
    Ps, cfg = oracle_sample(sample_frac)
    deg = cfg["sh_degree"]
    cam = cfg["cams"][0]
    target = np.zeros((3, cam.height, cam.width))
    W_, M_, V_ = Ps.copy(), np.zeros_like(Ps), np.zeros_like(Ps)
    C_ = np.zeros(Ps.shape[1], np.uint8)
    hp = orc.AdamHyper(lr=1e-3, eps=1e-15)
    t0 = time.perf_counter()
    for s in range(steps):
        _oracle_step(orc, Ps, deg, cam, target, W_, M_, V_, C_, s + 1, hp)
    dt = (time.perf_counter() - t0) / steps
    scale = 1.0 / sample_frac
    return {"value": round(1.0 / (dt * scale), 6), "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle step (cull+render+L1+backward+deferred Adam) on a random {sample_frac:.0%} of the "
                      f"10M Gaussians, one 1920x1080 view, {steps} step(s); time scaled linearly by "
                      f"{scale:.0f}x to the full Gaussian count",
            "seconds_per_sample_step": round(dt, 3)}


def run_oracle_workloads(args):
    """FP64 oracle timings on the host cores for every workload (a baseline for
    context, never a target): full steps of the 10k and 200k cases, the first
    three steps of the 1M orbit, one step of the 10M aerial workload and its
    cull and deferred Adam alone; single-threaded and on every core.  The 40M
    case is not run: its FP64 w, m, v alone need 57 GB.  One JSON line per
    (workload, threads)."""
    from oracle import oracle as orc
    from synth import scenes
    all_cores = orc.num_threads()
    hp = orc.AdamHyper(lr=1e-3, eps=1e-15)

    def cases():
        c = scenes.cfg_small_step()
        yield "cube10k_64px_sh0", c["scene"], c["target_scene"], c["cams"][:1], 0, False
        c = scenes.cfg_diff_check()
        yield "cube200k_512px_sh3", c["scene"], c["target_scene"], c["cams"][:1], 3, False
        c = scenes.cfg_heightfield_1m(n_views=3)
        yield "heightfield1m_1080p_sh3 (steps 1-3)", c["scene"], None, c["cams"][:3], 3, False
        c = scenes.cfg_aerial(n_views=1)
        yield WORKLOAD, c["scene"], None, c["cams"][:1], 3, True

    for name, P32, T32, cams, deg, split_stages in cases():
        P = np.ascontiguousarray(P32, np.float64)
        n = P.shape[1]
        for threads in (1, all_cores):
            orc.set_num_threads(threads)
            W_, M_, V_ = P.copy(), np.zeros_like(P), np.zeros_like(P)
            C_ = np.zeros(n, np.uint8)
            times, line = [], {"workload": name, "gaussians": n, "threads": threads, "impl": "reference",
                               "kind": "oracle"}
            for s, cam in enumerate(cams):
                target = (orc.render(np.asarray(T32, np.float64), deg, cam)["image"] if T32 is not None
                          else np.zeros((3, cam.height, cam.width)))
                t0 = time.perf_counter()
                _, n_vis = _oracle_step(orc, P, deg, cam, target, W_, M_, V_, C_, s + 1, hp)
                times.append(time.perf_counter() - t0)
            line.update(seconds_per_step=[round(t, 3) for t in times], visible=int(n_vis))
            if split_stages:
                # the cull (projection of every Gaussian) and the deferred update alone
                t0 = time.perf_counter()
                sp = orc.project(W_, deg, orc.camera(cams[0]))
                t_cull = time.perf_counter() - t0
                kept = np.nonzero(sp["keep"])[0].astype(np.int32)
                g = np.zeros((P.shape[0], kept.size))
                t0 = time.perf_counter()
                orc.adam_deferred(W_, M_, V_, C_, kept, g, len(cams) + 1, hp)
                t_adam = time.perf_counter() - t0
                line.update(cull_seconds=round(t_cull, 3), adam_seconds=round(t_adam, 3))
            print(json.dumps(line), flush=True)
        del P


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc
    frac = 0.02
    Ps, cfg = oracle_sample(frac)
    deg = cfg["sh_degree"]
    cams = cfg["cams"]
    W_, M_, V_ = Ps.copy(), np.zeros_like(Ps), np.zeros_like(Ps)
    C_ = np.zeros(Ps.shape[1], np.uint8)
    hp = orc.AdamHyper(lr=1e-3, eps=1e-15)
    target = np.zeros((3, cams[0].height, cams[0].width))
    for s in range(args.warmup):
        _oracle_step(orc, Ps, deg, cams[s % len(cams)], target, W_, M_, V_, C_, s + 1, hp)
    t0 = time.perf_counter()
    for s in range(args.steps):
        _oracle_step(orc, Ps, deg, cams[(args.warmup + s) % len(cams)], target, W_, M_, V_, C_,
                     args.warmup + s + 1, hp)
    dt = (time.perf_counter() - t0) / args.steps
    value = 1.0 / (dt / frac)
    sample = (f"FP64 oracle step on a random {frac:.0%} of the 10M Gaussians, one 1920x1080 view per step; "
              f"time scaled linearly by {1 / frac:.0f}x")
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 / value, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded aerial heightfield)", "impl": "reference",
           "config": {"workload": WORKLOAD, "gaussians": 10_000_000, "image": "1920x1080", "sh_degree": 3,
                      "views_per_step": 1, "form": "fp64 oracle"},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--gaussians", type=int, default=10_000_000)
    ap.add_argument("--views", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bf16", action="store_true", help="skip the bf16 precision-form measurement")
    ap.add_argument("--bf16-only", action="store_true",
                    help="time only the bf16 precision form (profiling); the JSON line then describes it")
    ap.add_argument("--density-of", type=int, default=None,
                    help="scale the scene area so that --gaussians keeps the density of this many (profiling cases)")
    ap.add_argument("--tile", default="8x4", help="raster tile WxH (W in 4..64, W*H in 32, 64, 128, 256)")
    ap.add_argument("--image", default="1920x1080", help="view size WxH")
    ap.add_argument("--views-per-step", type=int, default=1, help="views rendered and summed per training step")
    ap.add_argument("--budget-gb", type=float, default=None,
                    help="HBM budget: state that does not fit moves its SH planes to pinned host memory")
    ap.add_argument("--chunk-shift", type=int, default=11, help="log2 Gaussians per host-tier chunk")
    ap.add_argument("--cpu-optimizer", action="store_true",
                    help="the paper's offloaded configuration: SH planes in host memory stepped by the host cores")
    ap.add_argument("--cpu-threads", type=int, default=0, help="host-core optimizer threads (0: every core)")
    ap.add_argument("--raster-variant", default=None,
                    help="pin the rasterizer variant instead of the autotuned one: V, or F,B for forward and backward")
    ap.add_argument("--no-extra-forms", dest="extra_forms", action="store_false",
                    help="skip the batched-bf16 and 40M host-tier sub-records of the default line")
    ap.add_argument("--config-timings", action="store_true",
                    help="time the GPU path on the smaller workload definitions (10k step, 1M orbit, 200k fwd+bwd)")
    ap.add_argument("--split-demo", action="store_true",
                    help="measure balance-aware image splitting (§4.4) on a 1M-Gaussian view that crosses mem_limit")
    ap.add_argument("--oracle-workloads", action="store_true",
                    help="with --impl reference: time the FP64 oracle on every workload, 1 thread and all cores")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.split_demo:
        run_split_demo(args)
    elif args.config_timings:
        run_config_timings(args)
    elif args.impl == "reference" and args.oracle_workloads:
        run_oracle_workloads(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
