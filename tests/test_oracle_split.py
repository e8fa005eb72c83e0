"""Pins of the oracle's image splitting (GS-Scale §4.4): region counts on a
scene whose answer follows from where its Gaussians are placed, and the
balance search against brute force over every tile boundary."""
import math

import numpy as np
import pytest

from synth import scenes

C0 = 0.5 / math.sqrt(math.pi)
FX, W, H, Z = 100.0, 128, 32, 5.0
TILE = (8, 4)


def _point_scene(pixels):
    """Tiny isotropic Gaussians at depth Z whose centres project onto the
    given (x, y) pixel positions of a camera at the origin looking down +z.
    With scale 1e-4 the 2D covariance is the 0.3 low-pass alone, so
    lambda_max = 0.3 + sqrt(0.1) and the radius is ceil(3 sqrt(0.616)) = 3."""
    n = len(pixels)
    P = np.zeros((14, n))
    for i, (px, py) in enumerate(pixels):
        P[0, i] = (px - W / 2) * Z / FX
        P[1, i] = (py - H / 2) * Z / FX
        P[2, i] = Z
        P[3:6, i] = math.log(1e-4)
        P[6, i] = 1.0
        P[11:14, i] = (0.5 - 0.5) / C0
    return P


def _camera():
    return scenes.Camera(np.eye(3), np.zeros(3), FX, FX, W / 2, H / 2, W, H)


def test_region_counts_closed_form(orc):
    """Gaussian k sits at the centre of tile column c_k (radius 3 < 4, so its
    rectangle is that one column); one more straddles the boundary between
    columns 5 and 6.  Region counts at boundary `at`: #{c_k < at} + straddler
    if at <= 6 (it reaches column 5), #{c_k >= at} + straddler if at >= 6."""
    cols = [0, 1, 1, 3, 3, 3, 7, 8, 12, 15, 15]
    pixels = [(8 * c + 4, 14) for c in cols] + [(48.0, 14)]
    P = _point_scene(pixels)
    oc = orc.camera(_camera(), TILE)
    sp = orc.project(P, 0, oc)
    assert np.all(sp["keep"] == 1)
    assert np.all(sp["radius"] == 3)
    np.testing.assert_array_equal(sp["rect"][:-1, 0], cols)
    np.testing.assert_array_equal(sp["rect"][:-1, 1], np.array(cols) + 1)
    assert tuple(sp["rect"][-1, :2]) == (5, 7)
    tiles_x = orc.tiles_of(oc)[0]
    assert tiles_x == 16
    for at in range(1, tiles_x):
        first, second = orc.split_counts(sp, 0, at)
        assert first == sum(c < at for c in cols) + (at >= 6)
        assert second == sum(c >= at for c in cols) + (at <= 6)
    # along y every Gaussian lies in tile row 3 (pixel rows 12..15) or reaches row 4
    rows = sp["rect"][:, 2:]
    for at in range(1, orc.tiles_of(oc)[1]):
        first, second = orc.split_counts(sp, 1, at)
        assert first == int(np.sum(rows[:, 0] < at)) and second == int(np.sum(rows[:, 1] > at))


def _brute_force_boundary(orc, sp, axis, tiles):
    """The last inner boundary whose first region holds no more visible
    Gaussians than the second (1 if there is none): where bisection on the
    non-decreasing difference first - second converges."""
    best = 1
    for at in range(1, tiles):
        first, second = orc.split_counts(sp, axis, at)
        if first <= second:
            best = at
    return best


@pytest.mark.parametrize("seed,axis", [(31, 0), (32, 0), (33, 1), (34, 1)])
def test_balance_search_converges_to_brute_force(orc, seed, axis):
    """With enough steps (tiles <= 32 here, 5 halvings reach one boundary) the
    bisection returns the brute-force boundary; the count difference is
    non-decreasing in the boundary, which is what makes bisection valid."""
    P = scenes.uniform_cube_scene(4000, seed=seed, sh_degree=0, log_scale_mean=-3.0)
    P[0] = np.where(P[0] < 0.3, P[0], P[0] * 0.2)          # a denser band: the balance point is off-centre
    cam = scenes.camera_lookat((0.2, -0.1, -3.0), (0.0, 0.0, 0.0), 128, 96, 60.0, up=(0, -1, 0))
    oc = orc.camera(cam, TILE)
    sp = orc.project(P, 0, oc)
    tiles = orc.tiles_of(oc)[axis]
    assert tiles <= 32
    diffs = [np.subtract(*orc.split_counts(sp, axis, at)) for at in range(1, tiles)]
    assert all(b >= a for a, b in zip(diffs, diffs[1:]))
    at, counts = orc.balance_split(sp, oc, axis, steps=5)
    assert at == _brute_force_boundary(orc, sp, axis, tiles)
    assert counts == orc.split_counts(sp, axis, at)
    n_vis = int(np.sum(sp["keep"] == 1))
    assert counts[0] + counts[1] >= n_vis       # straddlers count twice


def test_five_steps_bracket_the_balance_point(orc):
    """At the benchmark's width (1920 px, 8-px tiles: 240 boundaries) five
    halvings leave an interval of 7.5 tiles: the result lies within 8 tiles
    of the brute-force boundary."""
    P = scenes.uniform_cube_scene(6000, seed=35, sh_degree=0, log_scale_mean=-3.0)
    P[0] = np.where(P[0] > -0.4, P[0], P[0] * 0.3)
    cam = scenes.camera_lookat((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 1920, 64, 60.0, up=(0, -1, 0))
    oc = orc.camera(cam, TILE)
    sp = orc.project(P, 0, oc)
    tiles = orc.tiles_of(oc)[0]
    assert tiles == 240
    at, _ = orc.balance_split(sp, oc, 0, steps=5)
    assert abs(at - _brute_force_boundary(orc, sp, 0, tiles)) <= 8
    at_full, _ = orc.balance_split(sp, oc, 0, steps=9)      # 2^8 >= 240: converged
    assert at_full == _brute_force_boundary(orc, sp, 0, tiles)
