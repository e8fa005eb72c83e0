"""Pins of the oracle's renderer (GS-Scale §2.4 steps 1-5) against things
other than itself: closed forms, library routines, brute force, finite
differences and mathematical invariants."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from synth import scenes

C0 = 0.5 / math.sqrt(math.pi)


def _one_gaussian_params(means, log_scales, quats, opac_logits, rgbs, deg=0):
    n = len(means)
    D = 11 + 3 * (deg + 1) ** 2
    P = np.zeros((D, n))
    for i in range(n):
        P[0:3, i] = means[i]
        P[3:6, i] = log_scales[i]
        P[6:10, i] = quats[i]
        P[10, i] = opac_logits[i]
        P[11:14, i] = (np.asarray(rgbs[i]) - 0.5) / C0
    return P


def _axis_camera(W=32, H=32):
    return scenes.camera_from_pose(np.eye(3), np.zeros(3), W, H, 60.0)


def _closed_form_alpha(f, s, z, o, W, H):
    """One isotropic Gaussian on the optical axis: Sigma2 = ((f s / z)^2 + 0.3) I,
    centred on the principal point; alpha = min(0.999, o exp(-|d|^2 / (2 var)))."""
    var = (f * s / z) ** 2 + 0.3
    r = math.ceil(3 * math.sqrt(var + math.sqrt(0.1)))   # lambda_max = var + sqrt(max(0.1, 0))
    px = np.arange(W) + 0.5
    py = np.arange(H) + 0.5
    dx = W / 2 - px[None, :]
    dy = H / 2 - py[:, None]
    raw = o * np.exp(-(dx ** 2 + dy ** 2) / (2 * var))
    alpha = np.minimum(0.999, raw)
    inside = (np.abs(dx) <= r) & (np.abs(dy) <= r) & (alpha >= 1 / 255)
    return np.where(inside, alpha, 0.0), r, var


@pytest.mark.parametrize("logit,ls", [(0.3, math.log(0.34)), (10.0, math.log(0.2)), (-2.0, math.log(0.6))])
def test_single_isotropic_closed_form(orc, logit, ls):
    cam = _axis_camera()
    rgb = (0.2, 0.7, 0.45)
    z = 5.0
    P = _one_gaussian_params([(0, 0, z)], [(ls,) * 3], [(1, 0, 0, 0)], [logit], [rgb])
    r = orc.render(P, 0, cam)
    o = 1 / (1 + math.exp(-logit))
    alpha, rad, var = _closed_form_alpha(cam.fx, math.exp(ls), z, o, 32, 32)
    sp = r["splats"][0]
    assert sp["keep"] == 1
    assert sp["radius"] == rad
    np.testing.assert_allclose(sp["cov2d"], [var, 0.0, var], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(sp["conic"], [1 / var, 0.0, 1 / var], rtol=1e-13)
    np.testing.assert_allclose(sp["mean2d"], [16.0, 16.0], atol=1e-12)
    expect = np.stack([c * alpha for c in rgb])
    np.testing.assert_allclose(r["image"], expect, atol=1e-12)


def test_two_gaussians_on_axis(orc):
    """C = c1 a1 + c2 a2 (1 - a1): the nearer Gaussian is composited first,
    whatever its index."""
    cam = _axis_camera()
    c_far, c_near = (0.9, 0.1, 0.3), (0.2, 0.8, 0.5)
    P = _one_gaussian_params([(0, 0, 7.0), (0, 0, 4.0)], [(math.log(0.5),) * 3, (math.log(0.25),) * 3],
                             [(1, 0, 0, 0)] * 2, [1.0, 0.0], [c_far, c_near])
    r = orc.render(P, 0, cam)
    a_far, _, _ = _closed_form_alpha(cam.fx, 0.5, 7.0, 1 / (1 + math.exp(-1.0)), 32, 32)
    a_near, _, _ = _closed_form_alpha(cam.fx, 0.25, 4.0, 0.5, 32, 32)
    expect = np.stack([cn * a_near + cf * a_far * (1 - a_near) for cn, cf in zip(c_near, c_far)])
    np.testing.assert_allclose(r["image"], expect, atol=1e-12)


def test_transmittance_stop(orc):
    """Nearly opaque layers: compositing stops before the layer that would take
    T below 1e-4 (alpha ~ 0.95: T = 1, 0.05, 0.0025, 1.25e-4, then stop)."""
    cam = _axis_camera()
    n = 6
    logit = math.log(0.95 / 0.05)
    depths = [3.0 + k for k in range(n)]
    P = _one_gaussian_params([(0, 0, z) for z in depths], [(math.log(2.0),) * 3] * n,
                             [(1, 0, 0, 0)] * n, [logit] * n, [(1.0, 0.5, 0.25)] * n)
    r = orc.render(P, 0, cam)
    alphas = [_closed_form_alpha(cam.fx, 2.0, z, 0.95, 32, 32)[0][16, 16] for z in depths]
    T, acc, used = 1.0, 0.0, 0
    for a in alphas:
        if T * (1 - a) < 1e-4:
            break
        acc += a * T
        T *= 1 - a
        used += 1
    assert used == 3
    np.testing.assert_allclose(r["image"][:, 16, 16], np.array([1.0, 0.5, 0.25]) * acc, rtol=1e-12)
    assert r["n_contrib"][16, 16] == 3
    np.testing.assert_allclose(r["T_final"][16, 16], T, rtol=1e-12)


def test_projection_against_library_rotation_and_numeric_jacobian(orc):
    """Sigma2 = J W Sigma3 W^T J^T + 0.3 I with Sigma3 built by scipy's
    quaternion->matrix routine and J by central differences of the pinhole map."""
    rng = np.random.default_rng(7)
    Rw = Rotation.random(random_state=3).as_matrix()
    cam = scenes.camera_from_pose(Rw, rng.normal(0, 0.3, 3) + np.array([0, 0, 6.0]), 96, 64, 70.0)
    n = 40
    pc = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.0, 1.0, n), rng.uniform(3, 9, n)])
    means = (Rw.T @ (pc - cam.t[:, None])).T          # world points that land in front of the camera
    quats = rng.normal(size=(n, 4))
    ls = rng.normal(-1.5, 0.5, (n, 3))
    P = _one_gaussian_params(means, ls, quats, np.zeros(n), [(0.5, 0.5, 0.5)] * n)
    sp = orc.project(P, 0, orc.camera(cam))

    def pix(mu):
        p = Rw @ mu + cam.t
        return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

    for i in range(n):
        qw, qx, qy, qz = quats[i]
        Rq = Rotation.from_quat([qx, qy, qz, qw]).as_matrix()   # scipy: scalar-last
        S3 = Rq @ np.diag(np.exp(2 * ls[i])) @ Rq.T
        h = 1e-5
        Jn = np.stack([(pix(means[i] + h * e) - pix(means[i] - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        S2 = Jn @ S3 @ Jn.T + 0.3 * np.eye(2)
        assert sp[i]["clampx"] == 0 and sp[i]["clampy"] == 0
        np.testing.assert_allclose(sp[i]["cov2d"], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose(sp[i]["mean2d"], pix(means[i]), rtol=1e-13)
        np.testing.assert_allclose(sp[i]["depth"], (Rw @ means[i] + cam.t)[2], rtol=1e-13)
        a, b, c = S2[0, 0], S2[0, 1], S2[1, 1]
        lam = 0.5 * (a + c) + math.sqrt(max(0.1, 0.25 * (a + c) ** 2 - (a * c - b * b)))
        assert sp[i]["radius"] == math.ceil(3 * math.sqrt(lam))
        np.testing.assert_allclose(np.array([[sp[i]["conic"][0], sp[i]["conic"][1]],
                                             [sp[i]["conic"][1], sp[i]["conic"][2]]]) @ S2, np.eye(2),
                                   atol=1e-7)


def _sphere_quadrature(nt=24, nph=48):
    x, w = np.polynomial.legendre.leggauss(nt)
    ph = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    ct = np.repeat(x, nph)
    st = np.sqrt(1 - ct ** 2)
    phi = np.tile(ph, nt)
    dirs = np.stack([st * np.cos(phi), st * np.sin(phi), ct], axis=1)
    wts = np.repeat(w, nph) * (2 * np.pi / nph)
    return dirs, wts


def test_sh_basis_signs_and_order_against_scipy(orc):
    """Signs and order of the 16 basis functions: the real spherical harmonics
    built from scipy's complex ones (Condon-Shortley phase included) as
    sqrt(2) Im Y_l^|m| for m < 0, Y_l^0, sqrt(2) Re Y_l^m for m > 0, in the
    order l = 0..3, m = -l..l (the convention of 3DGS colour coefficients),
    at random directions; and each degree's truncation (deg < 3 leaves the
    higher functions zero)."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(21)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(float(np.clip(d[2], -1.0, 1.0))), math.atan2(d[1], d[0])
        want = []
        for l in range(4):
            for m in range(-l, l + 1):
                y = complex(sph_harm_y(l, abs(m), theta, phi))
                want.append(math.sqrt(2.0) * y.imag if m < 0 else (y.real if m == 0 else math.sqrt(2.0) * y.real))
        for deg in range(4):
            Y, _ = orc.sh_basis(deg, d)
            k = (deg + 1) ** 2
            np.testing.assert_allclose(Y[:k], want[:k], rtol=0, atol=1e-12)
            assert np.all(Y[k:] == 0.0)


def test_sh_basis_orthonormal_and_harmonic(orc):
    """The 16 real SH functions are orthonormal on the sphere; each Y of degree l
    extends to a harmonic homogeneous polynomial |x|^l Y(x/|x|); dY matches
    central differences."""
    dirs, wts = _sphere_quadrature()
    Y = np.stack([orc.sh_basis(3, d)[0] for d in dirs])
    G = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)
    degree = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7)
    rng = np.random.default_rng(0)

    def solid(x, k):
        r = np.linalg.norm(x)
        return r ** degree[k] * orc.sh_basis(3, x / r)[0][k]

    for _ in range(5):
        x0 = rng.normal(size=3)
        x0 /= np.linalg.norm(x0)
        h = 1e-3
        for k in range(16):
            lap = sum(solid(x0 + h * e, k) + solid(x0 - h * e, k) - 2 * solid(x0, k) for e in np.eye(3)) / h ** 2
            assert abs(lap) < 1e-5
        # every Y_k is a homogeneous polynomial, so solid_k IS that polynomial and
        # dY (derivatives in x, y, z taken independently) is its gradient
        Yp, dY = orc.sh_basis(3, x0)
        h = 1e-6
        for k in range(16):
            grad_num = np.array([(solid(x0 + h * e, k) - solid(x0 - h * e, k)) / (2 * h) for e in np.eye(3)])
            np.testing.assert_allclose(dY[k], grad_num, atol=1e-8)
    # sh degree 0: rgb = Y00 * DC + 0.5 reproduces the colour the DC encodes
    assert abs(orc.sh_basis(0, np.array([0, 0, 1.0]))[0][0] - C0) < 1e-16


def _tiny_scene(seed, n=150, deg=0, W=32, H=24):
    P = scenes.uniform_cube_scene(n, seed=seed, sh_degree=deg, log_scale_mean=-2.2, log_scale_std=0.6,
                                  morton=False).astype(np.float64)
    rng = np.random.default_rng(seed)
    eye = rng.normal(0, 0.3, 3) + np.array([0.0, 0.0, -3.2])
    cam = scenes.camera_lookat(eye, rng.normal(0, 0.2, 3), W, H, 65.0, up=(0, -1, 0))
    return P, cam


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_equals_tiled(orc, seed):
    P, cam = _tiny_scene(seed, deg=1)
    brute = None
    for tile in [(16, 16), (8, 8), (16, 8), (32, 32), (4, 12)]:
        r = orc.render(P, 1, cam, tile=tile)
        b = orc.composite_brute(r["splats"], r["cam"])
        np.testing.assert_allclose(r["image"], b, atol=1e-12, rtol=0)
        if brute is None:
            brute = b
        np.testing.assert_allclose(r["image"], brute, atol=1e-12, rtol=0)
    assert r["n_contrib"].max() > 3


def _composite_untruncated(sp, P, W, H):
    """Per pixel, every Gaussian that survives the 3D cull with a positive
    determinant, in (FP32 depth, id) order, with the alpha floor, the 0.999
    clamp and the transmittance stop but without the 3-sigma square (nor the
    2D cull that follows from it).  Degree-0 colours and opacities straight
    from the parameters.  Returns the image and, per pixel, the summed alpha of
    the contributions the square test drops, and their largest alpha / o."""
    ok = np.isfinite(sp["conic"][:, 0]) & (sp["depth"] > 0.01) & (sp["cov2d"][:, 0] * sp["cov2d"][:, 2] -
                                                                  sp["cov2d"][:, 1] ** 2 > 0)
    ids = np.nonzero(ok)[0]
    order = ids[np.lexsort((ids, sp["depth_f32"][ids]))]
    o = 1.0 / (1.0 + np.exp(-P[10]))
    rgb = np.maximum(P[11:14] * C0 + 0.5, 0.0)
    img = np.zeros((3, H, W))
    dropped = np.zeros((H, W))
    worst = 0.0
    for py in range(H):
        for px in range(W):
            T = 1.0
            for i in order:
                dx, dy = px + 0.5 - sp["mean2d"][i, 0], py + 0.5 - sp["mean2d"][i, 1]
                A, B, Cc = sp["conic"][i]
                sig = 0.5 * (A * dx * dx + Cc * dy * dy) + B * dx * dy
                if sig < 0:
                    continue
                a = min(0.999, o[i] * math.exp(-sig))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                r = sp["radius"][i]
                if not (sp["keep"][i] and abs(dx) <= r and abs(dy) <= r):
                    dropped[py, px] += a
                    worst = max(worst, a / o[i])
                img[:, py, px] += rgb[:, i] * a * T
                T *= 1 - a
    return img, dropped, worst


@pytest.mark.parametrize("seed", [0, 1])
def test_truncation_error_of_the_3sigma_square(orc, seed):
    """Informational: the 3-sigma square drops contributions with sigma >= 4.5
    (outside the square |d| > r >= 3 sqrt(lambda_max)), so each dropped alpha
    is at most o e^-4.5, and the image moves by at most about twice the
    colour-weighted sum of the dropped alphas (their own share plus the
    transmittance they take from what lies behind) plus the stop tolerance."""
    P, cam = _tiny_scene(seed, n=60, deg=0, W=24, H=16)
    P[3:6] += 0.8                                   # larger splats: more of them reach past their squares
    r = orc.render(P, 0, cam, tile=(8, 8))
    img, dropped, worst = _composite_untruncated(r["splats"], P, cam.width, cam.height)
    assert worst <= math.exp(-4.5) * (1 + 1e-12), worst
    cmax = float(np.maximum(P[11:14] * C0 + 0.5, 0.0).max())
    err = np.abs(img - r["image"]).max(axis=0)
    assert np.all(err <= 2 * cmax * dropped + 2e-4 * cmax + 1e-12), float((err - 2 * cmax * dropped).max())
    print(f"3-sigma truncation: max |untruncated - tiled| = {err.max():.3e}, pixels affected "
          f"{np.mean(dropped > 0):.1%}")


def test_sort_against_library_lexsort(orc):
    P, cam = _tiny_scene(5, n=200)
    r = orc.render(P, 0, cam, tile=(8, 8))
    sp = r["splats"]
    tx, _ = orc.tiles_of(r["cam"])
    tiles, bits, gids = [], [], []
    for i in np.nonzero(sp["keep"])[0]:
        x0, x1, y0, y1 = sp["rect"][i]
        for ty in range(y0, y1):
            for txx in range(x0, x1):
                tiles.append(ty * tx + txx)
                bits.append(np.float32(sp["depth"][i]).view(np.uint32))
                gids.append(i)
    tiles, bits, gids = map(np.asarray, (tiles, bits, gids))
    # the pairs the Gaussian can reach (the list filter, pinned on its own below)
    reach = orc.tile_reach(sp, r["cam"], gids, tiles) >= 1 / 255
    assert 0 < reach.sum() < len(reach)
    tiles, bits, gids = tiles[reach], bits[reach], gids[reach]
    order = np.lexsort((gids, bits, tiles))
    np.testing.assert_array_equal(r["key_tile"], tiles[order])
    np.testing.assert_array_equal(r["key_gid"], gids[order])
    # ranges partition the sorted list per tile
    for t in range(r["ranges"].shape[0]):
        b, e = r["ranges"][t]
        assert np.all(r["key_tile"][b:e] == t)
        assert e - b == np.count_nonzero(tiles == t)


def _reach_by_sampling(sp, i, tile, tiles_x, tw, th, ext, m=241):
    """o exp(-sigma) maximised over an m x m grid of the box of the tile's pixel
    centres cut to the (widened) 3-sigma square, plus its corners."""
    mx, my = sp["mean2d"][i]
    r = sp["radius"][i] + ext
    X0 = (tile % tiles_x) * tw + 0.5
    Y0 = (tile // tiles_x) * th + 0.5
    x0, x1 = max(X0, mx - r), min(X0 + tw - 1, mx + r)
    y0, y1 = max(Y0, my - r), min(Y0 + th - 1, my + r)
    if x0 > x1 or y0 > y1:
        return 0.0
    xs, ys = np.linspace(x0, x1, m), np.linspace(y0, y1, m)
    dx = (mx - xs)[None, :]
    dy = (my - ys)[:, None]
    A, B, Cc = sp["conic"][i]
    sig = 0.5 * (A * dx * dx + Cc * dy * dy) + B * dx * dy
    return float(sp["opacity"][i] * np.exp(-sig.min()))


@pytest.mark.parametrize("tile", [(8, 8), (16, 4), (4, 8)])
def test_tile_reach_against_sampling(orc, tile):
    """The list filter's quantity -- the largest o exp(-sigma) over the part of
    a tile that the Gaussian's square covers -- against a dense grid: never
    below any sampled value, and within the grid's resolution of the largest.
    Anisotropic splats near tile corners, where the minimiser lies inside an
    edge, make a dropped or mis-signed cross term B visible."""
    P, cam = _tiny_scene(7, n=200)
    P[3:6] += np.random.default_rng(7).normal(0, 0.6, (3, P.shape[1]))
    r = orc.render(P, 0, cam, tile=tile)
    sp, oc = r["splats"], r["cam"]
    tx, _ = orc.tiles_of(oc)
    pairs = []
    for i in np.nonzero(sp["keep"])[0]:
        x0, x1, y0, y1 = sp["rect"][i]
        for ty in range(y0, y1):
            for txx in range(x0, x1):
                pairs.append((i, ty * tx + txx))
    pairs = np.asarray(pairs)
    rng = np.random.default_rng(1)
    pairs = pairs[rng.choice(len(pairs), size=min(400, len(pairs)), replace=False)]
    for ext in (0.0, 0.7):
        got = orc.tile_reach(sp, oc, pairs[:, 0], pairs[:, 1], ext=ext)
        ref = np.array([_reach_by_sampling(sp, i, t, tx, tile[0], tile[1], ext) for i, t in pairs])
        assert np.all(got >= ref * (1 - 1e-12)), np.max(ref - got)
        assert np.all(got <= ref * (1 + 2e-3) + 1e-300), np.max(got / np.maximum(ref, 1e-300))
        o = sp["opacity"][pairs[:, 0]]
        assert np.any(got == o) and np.any((got > 0) & (got < o))   # mean inside the box, and outside


def test_lists_hold_every_contributing_pair(orc):
    """Every (tile, Gaussian) whose tile has a pixel centre where the per-pixel
    rule lets the Gaussian contribute (square test, alpha >= 1/255) is in the
    oracle's lists, found by brute force over all pixels; and the filter does
    drop pairs of the rectangles (the rule has an effect here)."""
    P, cam = _tiny_scene(8, n=200)
    tile = (8, 4)
    r = orc.render(P, 0, cam, tile=tile)
    sp = r["splats"]
    tx, _ = orc.tiles_of(r["cam"])
    listed = set(zip(r["key_tile"].tolist(), r["key_gid"].tolist()))
    H, W = cam.height, cam.width
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    n_rect = 0
    for i in np.nonzero(sp["keep"])[0]:
        mx, my = sp["mean2d"][i]
        A, B, Cc = sp["conic"][i]
        dx, dy = xs - mx, ys - my
        sig = 0.5 * (A * dx * dx + Cc * dy * dy) + B * dx * dy
        alpha = np.minimum(0.999, sp["opacity"][i] * np.exp(-sig))
        rr = sp["radius"][i]
        ok = (np.abs(dx) <= rr) & (np.abs(dy) <= rr) & (alpha >= 1 / 255)
        for py, px in zip(*np.nonzero(ok)):
            assert ((py // tile[1]) * tx + px // tile[0], i) in listed
        x0, x1, y0, y1 = sp["rect"][i]
        n_rect += (x1 - x0) * (y1 - y0)
    assert len(listed) < n_rect


def test_cull_rules_and_special_cases(orc):
    cam = _axis_camera(64, 48)
    means = [(0, 0, -2.0),        # behind the camera
             (0, 0, 0.005),       # in front but before the near plane
             (30.0, 0, 5.0),      # far outside the image, small
             (3.5, 0, 5.0),       # centre off-screen, huge: overlaps the image
             (0.5, 0.2, 5.0)]     # plainly visible
    ls = [(math.log(0.1),) * 3, (math.log(0.1),) * 3, (math.log(0.1),) * 3, (math.log(1.5),) * 3,
          (math.log(0.1),) * 3]
    P = _one_gaussian_params(means, ls, [(1, 0, 0, 0)] * 5, [0.0] * 5, [(0.5,) * 3] * 5)
    sp = orc.project(P, 0, orc.camera(cam))
    np.testing.assert_array_equal(sp["keep"], [0, 0, 0, 1, 1])
    assert sp[3]["mean2d"][0] > 64                        # centre off to the right
    # generic rule on a random scene: kept <=> near < z < far and the 3-sigma
    # square [mu - r, mu + r] overlaps the tiled image area
    P, cam = _tiny_scene(11, n=400, W=48, H=40)
    P[0:3] *= 3.0                                         # spread the cube beyond the view and behind the camera
    oc = orc.camera(cam, (16, 8))
    sp = orc.project(P, 0, oc)
    tx, ty = orc.tiles_of(oc)
    zin = (sp["depth"] > cam.near) & (sp["depth"] < cam.far)
    mx, my, r = sp["mean2d"][:, 0], sp["mean2d"][:, 1], sp["radius"]
    overlap = (mx + r > 0) & (mx - r < tx * 16) & (my + r > 0) & (my - r < ty * 8)
    np.testing.assert_array_equal(sp["keep"].astype(bool), zin & overlap)
    assert 50 < sp["keep"].sum() < 350 and (~zin).sum() > 10


def test_l1_loss(orc):
    rng = np.random.default_rng(1)
    a, b = rng.random((3, 8, 8)), rng.random((3, 8, 8))
    b[0, 0, 0] = a[0, 0, 0]
    loss, d = orc.loss_l1(a, b)
    assert abs(loss - np.mean(np.abs(a - b))) < 1e-15
    np.testing.assert_array_equal(d, np.sign(a - b) / a.size)


def _fd_case(orc, P, deg, cam, weights, samples, h, tile=(8, 8)):
    base = orc.render(P, deg, cam, tile=tile)
    grad, _ = orc.backward(P, deg, base["cam"], base["splats"], base["key_gid"], base["ranges"], weights)
    keys = ("keep", "rect", "radius", "rgb_clamped", "clampx", "clampy")
    out, flagged = [], 0
    for (row, i) in samples:
        vals = []
        same = True
        for sgn in (+1, -1):
            Q = P.copy()
            Q[row, i] += sgn * h
            r = orc.render(Q, deg, cam, tile=tile)
            same &= bool(np.array_equal(r["decision_hash"], base["decision_hash"]))
            same &= all(np.array_equal(r["splats"][k], base["splats"][k]) for k in keys)
            vals.append(float(np.sum(weights * r["image"])))
        if not same:
            flagged += 1
            continue
        out.append(((vals[0] - vals[1]) / (2 * h), grad[row, i]))
    return np.array(out), flagged, grad


@pytest.mark.parametrize("deg,seed", [(0, 21), (3, 22)])
def test_adjoint_against_central_differences(orc, deg, seed):
    """The hand-derived adjoint equals central differences of <w, image(P)>
    for a fixed random weight image w (so no kink of the loss enters)."""
    P = scenes.uniform_cube_scene(80, seed=seed, sh_degree=deg, log_scale_mean=-1.8, log_scale_std=0.4,
                                  degenerate_frac=0.1, morton=False).astype(np.float64)
    P[11 + 3:, :] *= 20.0                              # make view-dependent colour matter
    cam = scenes.camera_lookat((0.3, -0.2, -3.0), (0.0, 0.1, 0.0), 24, 20, 70.0, up=(0, -1, 0))
    rng = np.random.default_rng(seed)
    wimg = rng.normal(size=(3, 20, 24))
    sp = orc.project(P, deg, orc.camera(cam, (8, 8)))
    kept = np.nonzero(sp["keep"])[0]
    D = P.shape[0]
    samples = [(int(rng.integers(0, D)), int(rng.choice(kept))) for _ in range(250)]
    res, flagged, grad = _fd_case(orc, P, deg, cam, wimg, samples, h=1e-5)
    assert flagged < 0.2 * len(samples)
    fd, ad = res[:, 0], res[:, 1]
    scale = np.abs(grad).max()
    err = np.abs(fd - ad) / (np.abs(ad) + 1e-6 * scale)
    assert np.count_nonzero(np.abs(ad) > 1e-6 * scale) > 100
    assert err.max() < 1e-5, (err.max(), np.argmax(err))


def test_l1_gradient_is_chain_of_adjoint(orc):
    """dL/dP for the L1 loss equals the adjoint applied to sign(C - C_gt)/(3HW),
    checked by central differences of the loss itself."""
    P, cam = _tiny_scene(31, n=60, deg=0, W=16, H=16)
    tgt = orc.render(_tiny_scene(32, n=60, deg=0, W=16, H=16)[0], 0, cam)["image"]
    r = orc.render_loss_backward(P, 0, cam, tgt, tile=(8, 8))
    rng = np.random.default_rng(3)
    kept = np.nonzero(r["splats"]["keep"])[0]
    checked = 0
    for _ in range(60):
        row, i = int(rng.integers(0, 14)), int(rng.choice(kept))
        h = 1e-6
        lv = []
        ok = True
        for s in (1, -1):
            Q = P.copy()
            Q[row, i] += s * h
            rq = orc.render(Q, 0, cam, tile=(8, 8))
            ok &= np.array_equal(rq["decision_hash"], r["decision_hash"])
            ok &= np.array_equal(np.sign(rq["image"] - tgt), np.sign(r["image"] - tgt))
            lv.append(orc.loss_l1(rq["image"], tgt)[0])
        if not ok:
            continue
        fd = (lv[0] - lv[1]) / (2 * h)
        g = r["grad"][row, i]
        assert abs(fd - g) <= 1e-5 * abs(g) + 1e-10, (row, i, fd, g)   # FD rounding floor ~ eps(L)/h
        checked += 1
    assert checked > 30
