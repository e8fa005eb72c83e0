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


def _scene_in_one_block(n, seed):
    """The heightfield recipe drawn the direct way (the SH block in one draw,
    then one Morton gather), against which the streamed generator is checked."""
    rng = np.random.Generator(np.random.PCG64(seed))
    e, A, (lx, ly), ncl, csz = 50.0, 5.0, (20.0, 25.0), 2, 2000
    n_cl = min(n, ncl * csz)
    n_gr = n - n_cl
    gx, gy = rng.uniform(-e, e, n_gr), rng.uniform(-e, e, n_gr)
    gz = A * np.sin(gx / lx) * np.cos(gy / ly) + rng.normal(0.0, 0.5, n_gr)
    cx, cy = rng.uniform(-e, e, ncl), rng.uniform(-e, e, ncl)
    cz = A * np.sin(cx / lx) * np.cos(cy / ly) + rng.uniform(0.0, 20.0, ncl)
    which = np.repeat(np.arange(ncl), csz)[:n_cl]
    px, py, pz = (c[which] + rng.normal(0.0, 2.0, n_cl) for c in (cx, cy, cz))
    means = np.stack([np.concatenate([gx, px]), np.concatenate([gy, py]), np.concatenate([gz, pz])])
    ls = np.concatenate([rng.normal(math.log(0.2), 0.3, (3, n_gr)), rng.normal(math.log(0.1), 0.3, (3, n_cl))], axis=1)
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    opac = rng.standard_normal(n)
    sh = np.empty((16, 3, n))
    sh[0] = (rng.uniform(0.0, 1.0, (3, n)) - 0.5) * scenes.DC_FROM_RGB
    sh[1:] = rng.normal(0.0, 0.01, (15, 3, n))
    p = np.concatenate([means, ls, q, opac[None], sh.reshape(48, n)]).astype(np.float32)
    return p[:, scenes.morton_order(means)]


def test_streamed_generator_equals_one_block_draw():
    got = scenes.heightfield_scene(30_000, seed=5, half_extent=50.0, n_clusters=2, cluster_size=2000, sh_degree=3)
    np.testing.assert_array_equal(got, _scene_in_one_block(30_000, 5))
