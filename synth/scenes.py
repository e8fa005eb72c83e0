"""Seeded scene and camera generators.

Layout of a scene (a "Gaussian set"): one float32 array ``params`` of shape
[D][n] (structure of arrays), rows

    0..2    mean x, y, z                      (world units)
    3..5    log-scale x, y, z
    6..9    quaternion w, x, y, z             (not normalised)
    10      opacity logit
    11..    SH coefficients, coefficient-major: row 11 + 3*k + c is
            coefficient k (0..(L+1)^2-1) of colour channel c

so D = 11 + 3*(L+1)^2: 14 for SH degree 0, 59 for degree 3 (the 59 parameters
of §2.3).  Gaussians are stored in Morton (Z-curve) order of their means so
that the Gaussians one view sees form long index runs.

Cameras are OpenCV pinhole cameras (x right, y down, z forward) given as a
world-to-camera rotation R (row-major 3x3) and translation t, focal lengths
fx, fy, principal point cx, cy, near/far depths and the image size.  A field
of view is read as horizontal: fx = fy = (W/2)/tan(fov/2), cx = W/2, cy = H/2.

Nothing here evaluates the method: these functions only draw random numbers
(numpy PCG64) and arrange them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from concurrent.futures import ThreadPoolExecutor

import numpy as np

__all__ = [
    "ROW_MEAN", "ROW_LOGSCALE", "ROW_QUAT", "ROW_OPACITY", "ROW_SH",
    "n_params", "Camera", "camera_from_pose", "camera_lookat", "camera_aerial",
    "uniform_cube_scene", "heightfield_scene", "morton_order",
    "cfg_small_step", "cfg_heightfield_1m", "cfg_diff_check", "cfg_aerial",
    "orbit_cameras", "aerial_cameras", "DC_FROM_RGB",
]

ROW_MEAN, ROW_LOGSCALE, ROW_QUAT, ROW_OPACITY, ROW_SH = 0, 3, 6, 10, 11

# The zeroth real spherical harmonic is the constant 1/(2 sqrt(pi)).  A DC
# coefficient that renders as colour u (with the +0.5 offset of 3DGS) is
# (u - 0.5) / Y00; scene recipes that specify colours store them this way.
_Y00 = 0.5 / math.sqrt(math.pi)
DC_FROM_RGB = 1.0 / _Y00


def n_params(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


@dataclass
class Camera:
    R: np.ndarray            # (3, 3) float64 world -> camera rotation
    t: np.ndarray            # (3,) float64
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.01
    far: float = 1e10
    extra: dict = field(default_factory=dict)

    @property
    def center(self) -> np.ndarray:
        return -self.R.T @ self.t


def _intrinsics(width: int, height: int, fov_x_deg: float):
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return fx, fx, width / 2.0, height / 2.0


def camera_from_pose(R, t, width, height, fov_x_deg=60.0, near=0.01, far=1e10) -> Camera:
    fx, fy, cx, cy = _intrinsics(width, height, fov_x_deg)
    return Camera(np.asarray(R, np.float64).reshape(3, 3), np.asarray(t, np.float64).reshape(3),
                  fx, fy, cx, cy, int(width), int(height), near, far)


def camera_lookat(eye, target, width, height, fov_x_deg=60.0, up=(0.0, 0.0, 1.0),
                  near=0.01, far=1e10) -> Camera:
    """Camera at ``eye`` whose optical axis passes through ``target``."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    if np.linalg.norm(right) < 1e-9:           # looking straight along `up`
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    return camera_from_pose(R, -R @ eye, width, height, fov_x_deg, near, far)


def camera_aerial(eye, heading, pitch, width, height, fov_x_deg=60.0) -> Camera:
    """Aerial camera: ``heading`` (rad, about +z) and ``pitch`` (rad, -pi/2 = nadir)."""
    ch, sh = math.cos(heading), math.sin(heading)
    cp, sp = math.cos(pitch), math.sin(pitch)
    fwd = np.array([cp * ch, cp * sh, sp])
    right = np.array([sh, -ch, 0.0])
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    eye = np.asarray(eye, np.float64)
    return camera_from_pose(R, -R @ eye, width, height, fov_x_deg)


# ---------------------------------------------------------------- layout helpers

def _part1by2(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(xyz: np.ndarray) -> np.ndarray:
    """Permutation that sorts points (3, n) along a 21-bit-per-axis Z-curve."""
    lo = xyz.min(axis=1, keepdims=True)
    hi = xyz.max(axis=1, keepdims=True)
    q = ((xyz - lo) / np.maximum(hi - lo, 1e-12) * 2097151.0).astype(np.uint64)
    code = _part1by2(q[0]) | (_part1by2(q[1]) << np.uint64(1)) | (_part1by2(q[2]) << np.uint64(2))
    return np.argsort(code, kind="stable")


def _random_quats(rng, n):
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q


def _assemble(means, log_scales, quats, opac_logit, rng, n, sh_degree, morton=True, rest_std=0.01):
    """The [D][n] float32 scene: the 11 geometry rows, then the SH rows drawn
    from ``rng`` after everything else (DC from colours uniform in [0,1], the
    higher coefficients N(0, rest_std^2)), in Morton order of the means.  The
    SH rows are drawn one at a time (the same stream, in the same order, as one
    draw of the whole block) and written straight to their place, so a large
    scene never holds them in float64."""
    k = (sh_degree + 1) ** 2
    D = 11 + 3 * k
    order = morton_order(means) if morton else None
    p = np.empty((D, n), np.float32)
    step = max(1, -(-n // 8))
    with ThreadPoolExecutor(8) as gather_pool, ThreadPoolExecutor(1) as row_pool:
        def put(row, values):
            # the permutation gather in 8 slices on threads (numpy releases the GIL there)
            if not morton:
                p[row] = values
                return
            list(gather_pool.map(lambda a: p.__setitem__((row, slice(a, a + step)), values[order[a:a + step]]),
                                 range(0, n, step)))

        for r in range(3):
            put(r, means[r])
            put(3 + r, log_scales[r])
        for r in range(4):
            put(6 + r, quats[r])
        put(10, opac_logit)
        dc = (rng.uniform(0.0, 1.0, (3, n)) - 0.5) * DC_FROM_RGB
        for c in range(3):
            put(11 + c, dc[c])
        del dc
        pending = None
        for r in range(3, 3 * k):
            values = rng.normal(0.0, rest_std, n)          # the next row's draw overlaps the last row's gather
            if pending is not None:
                pending.result()
            pending = row_pool.submit(put, 11 + r, values)
        if pending is not None:
            pending.result()
    return p


# ---------------------------------------------------------------- scenes

def uniform_cube_scene(n, seed, sh_degree=0, log_scale_mean=-3.0, log_scale_std=0.5,
                       degenerate_frac=0.0, half_extent=1.0, morton=True):
    """Means uniform in [-e, e]^3, log-scales N(mu, sd^2), uniform random unit
    quaternions, opacity sigmoid(N(0,1)), colours uniform in [0,1].
    ``degenerate_frac`` of the Gaussians get one random axis at log-scale -9."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-half_extent, half_extent, (3, n))
    ls = rng.normal(log_scale_mean, log_scale_std, (3, n))
    if degenerate_frac > 0:
        nd = int(round(degenerate_frac * n))
        sel = rng.choice(n, nd, replace=False)
        ax = rng.integers(0, 3, nd)
        ls[ax, sel] = -9.0
    quats = _random_quats(rng, n)
    opac = rng.standard_normal(n)
    return _assemble(means, ls, quats, opac, rng, n, sh_degree, morton)


def heightfield_scene(n, seed, half_extent=100.0, amplitude=5.0, wavelength=(20.0, 25.0),
                      n_clusters=20, cluster_size=10_000, sh_degree=3, morton=True,
                      ground_log_scale=math.log(0.2), cluster_log_scale=math.log(0.1)):
    """Ground heightfield z = A sin(x/lx) cos(y/ly) + N(0, 0.5^2) over
    [-e, e]^2 plus Gaussian-distributed clusters (centres on the surface,
    lifted U[0, 20]; offsets N(0, 2^2))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_cl = min(n, n_clusters * cluster_size)
    n_gr = n - n_cl
    lx, ly = wavelength
    gx = rng.uniform(-half_extent, half_extent, n_gr)
    gy = rng.uniform(-half_extent, half_extent, n_gr)
    gz = amplitude * np.sin(gx / lx) * np.cos(gy / ly) + rng.normal(0.0, 0.5, n_gr)
    cx = rng.uniform(-half_extent, half_extent, n_clusters)
    cy = rng.uniform(-half_extent, half_extent, n_clusters)
    cz = amplitude * np.sin(cx / lx) * np.cos(cy / ly) + rng.uniform(0.0, 20.0, n_clusters)
    which = np.repeat(np.arange(n_clusters), cluster_size)[:n_cl]
    px = cx[which] + rng.normal(0.0, 2.0, n_cl)
    py = cy[which] + rng.normal(0.0, 2.0, n_cl)
    pz = cz[which] + rng.normal(0.0, 2.0, n_cl)
    means = np.stack([np.concatenate([gx, px]), np.concatenate([gy, py]), np.concatenate([gz, pz])])
    ls = np.concatenate([rng.normal(ground_log_scale, 0.3, (3, n_gr)),
                         rng.normal(cluster_log_scale, 0.3, (3, n_cl))], axis=1)
    quats = _random_quats(rng, n)
    opac = rng.standard_normal(n)
    return _assemble(means, ls, quats, opac, rng, n, sh_degree, morton)


def orbit_cameras(n_views, radius, altitude, width=1920, height=1080, fov_x_deg=60.0, phase=0.0):
    """Cameras on a circle of ``radius`` at ``altitude``, all looking at the origin."""
    cams = []
    for k in range(n_views):
        th = phase + 2.0 * math.pi * k / n_views
        cams.append(camera_lookat((radius * math.cos(th), radius * math.sin(th), altitude),
                                  (0.0, 0.0, 0.0), width, height, fov_x_deg))
    return cams


def aerial_cameras(n_views, seed, half_extent, alt=(150.0, 300.0), pitch_deg=(-90.0, -45.0),
                   width=1920, height=1080, fov_x_deg=60.0, margin=0.7):
    """Nadir-to-oblique aerial views over a square field."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cams = []
    for _ in range(n_views):
        x, y = rng.uniform(-margin * half_extent, margin * half_extent, 2)
        z = rng.uniform(*alt)
        pitch = math.radians(rng.uniform(*pitch_deg))
        heading = rng.uniform(0.0, 2.0 * math.pi)
        cams.append(camera_aerial((x, y, z), heading, pitch, width, height, fov_x_deg))
    return cams


# ---------------------------------------------------------------- named workloads

def cfg_small_step():
    """Plain FP32 single step: 10,000 Gaussians in [-1,1]^3, SH degree 0, one
    64x64 camera at z=-3 looking at the origin (fov 60 deg), 16x16 tiles;
    the target is rendered from the seed-1 scene."""
    scene = uniform_cube_scene(10_000, seed=0, sh_degree=0)
    target_scene = uniform_cube_scene(10_000, seed=1, sh_degree=0)
    cam = camera_from_pose(np.eye(3), (0.0, 0.0, 3.0), 64, 64, 60.0)
    return dict(name="cube10k_64px_sh0", scene=scene, target_scene=target_scene, cams=[cam],
                tile=(16, 16), sh_degree=0)


def cfg_heightfield_1m(n_views=100, orbit_radius=55.0, n=1_000_000):
    """1M Gaussians on a 200x200 m heightfield plus 20 clusters, SH degree 3,
    orbit of 1920x1080 cameras at 60 m altitude."""
    scene = heightfield_scene(n, seed=0)
    target_scene = heightfield_scene(n, seed=1)
    cams = orbit_cameras(n_views, orbit_radius, 60.0)
    return dict(name="heightfield1m_1080p_sh3", scene=scene, target_scene=target_scene,
                cams=cams, tile=(16, 16), sh_degree=3)


def cfg_diff_check(n=200_000, width=512):
    """Differentiation check: cube scene scaled down (log-scales N(-4, 0.5^2)),
    SH degree 3, 5% of Gaussians with one log-scale at -9, 512x512."""
    scene = uniform_cube_scene(n, seed=0, sh_degree=3, log_scale_mean=-4.0, degenerate_frac=0.05)
    target_scene = uniform_cube_scene(n, seed=1, sh_degree=3, log_scale_mean=-4.0, degenerate_frac=0.05)
    cam = camera_from_pose(np.eye(3), (0.0, 0.0, 3.0), width, width, 60.0)
    return dict(name="cube200k_512px_sh3", scene=scene, target_scene=target_scene, cams=[cam],
                tile=(16, 16), sh_degree=3)


def cfg_aerial(n=10_000_000, n_views=16, width=1920, height=1080, seed_views=2, scale=5.0,
               n_clusters=200):
    """Aerial heightfield: the 1M generator scaled x5 in x,y (1x1 km), 20 m
    amplitude, 200 clusters; nadir-oblique views at 150-300 m altitude.  A
    smaller n with scale 5 sqrt(n / 10M) and 200 n / 10M clusters keeps the 10M
    scene's density, hence the same per-view raster load."""
    he = 100.0 * scale
    scene = heightfield_scene(n, seed=0, half_extent=he, amplitude=20.0,
                              wavelength=(20.0 * scale, 25.0 * scale), n_clusters=n_clusters)
    cams = aerial_cameras(n_views, seed_views, he, width=width, height=height)
    return dict(name=f"aerial{n // 1_000_000}m_{height}p_sh3", scene=scene, cams=cams,
                tile=(16, 16), sh_degree=3, half_extent=he)
