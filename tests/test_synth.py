"""The seeded input generators: the Z-curve layout against a bit-by-bit
interleave, reproducibility from the seed, and the recipe's distributions."""
import math

import numpy as np

from synth import scenes


def _interleave_slow(x, y, z):
    code = 0
    for b in range(21):
        code |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
    return code


def test_morton_code_matches_bitwise_interleave():
    rng = np.random.default_rng(0)
    q = rng.integers(0, 1 << 21, size=(3, 500), dtype=np.uint64)
    fast = scenes._part1by2(q[0]) | (scenes._part1by2(q[1]) << np.uint64(1)) | (scenes._part1by2(q[2]) << np.uint64(2))
    for i in range(q.shape[1]):
        assert int(fast[i]) == _interleave_slow(int(q[0, i]), int(q[1, i]), int(q[2, i]))


def test_scene_is_morton_ordered_and_reproducible():
    a = scenes.uniform_cube_scene(20_000, seed=7, sh_degree=1)
    b = scenes.uniform_cube_scene(20_000, seed=7, sh_degree=1)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, scenes.uniform_cube_scene(20_000, seed=8, sh_degree=1))
    # stored order follows the Z-curve of the means: re-sorting is the identity
    np.testing.assert_array_equal(scenes.morton_order(a[0:3].astype(np.float64)), np.arange(a.shape[1]))


def test_cube_recipe_distributions():
    n = 200_000
    P = scenes.uniform_cube_scene(n, seed=3, sh_degree=3, log_scale_mean=-3.0, log_scale_std=0.5,
                                  degenerate_frac=0.05)
    assert P.shape == (59, n) and P.dtype == np.float32
    assert np.all(np.abs(P[0:3]) <= 1.0)
    q = P[6:10].astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(q, axis=0), 1.0, atol=1e-6)
    ls = P[3:6].astype(np.float64)
    degenerate = np.any(ls == -9.0, axis=0)
    assert abs(degenerate.mean() - 0.05) < 0.005
    normal = ls[:, ~degenerate]
    assert abs(normal.mean() + 3.0) < 0.01 and abs(normal.std() - 0.5) < 0.01
    # opacity sigmoid(N(0, 1)); degree-0 colours uniform in [0, 1] through the DC coefficient
    assert abs(P[10].mean()) < 0.01 and abs(P[10].std() - 1.0) < 0.01
    rgb = P[11:14].astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5
    assert rgb.min() >= -1e-6 and rgb.max() <= 1 + 1e-6 and abs(rgb.mean() - 0.5) < 0.01
