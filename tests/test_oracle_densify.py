"""Pins of the oracle's densification on a deferred-Adam state (§2.4 step 7
with the deferred update of §4.3): deferred training with densification
equals eager training with it, bit for bit with the replay catch-up; split
children, clones and pruning against closed forms."""
import math

import numpy as np

D = 14
LR = np.array([1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3, 1e-4])


def _params(rng, n):
    w = np.zeros((D, n))
    w[0:3] = rng.uniform(-1, 1, (3, n))
    w[3:6] = rng.normal(math.log(0.01), 0.6, (3, n))           # largest scales both sides of 0.01
    q = rng.normal(size=(4, n))
    w[6:10] = q / np.linalg.norm(q, axis=0)
    w[10] = rng.normal(0.0, 3.0, n)                            # some opacities below 0.005
    w[11:14] = rng.normal(0.0, 0.3, (3, n))
    return w


def _schedule(rng, n, steps):
    out = []
    for _ in range(steps):
        c = rng.integers(0, n)
        lo, hi = max(0, c - n // 5), min(n, c + n // 5)
        out.append(np.arange(lo, hi, dtype=np.int32))
    return out


def _train(orc, state, sched, grads, t0, hp, deferred):
    w, m, v, cnt = state
    n = w.shape[1]
    for k, ids in enumerate(sched):
        t = t0 + k + 1
        if deferred:
            orc.adam_deferred(w, m, v, cnt, ids, grads[k][:, ids], t, hp, mode=1)
        else:
            g = np.zeros((D, n))
            g[:, ids] = grads[k][:, ids]
            orc.adam_eager(w, m, v, g, t, hp)


def test_deferred_densify_equals_eager_densify(orc):
    """Train 20 steps, densify, train 15 more: the deferred run (replay
    catch-up), materialised, is the eager run bit for bit, with the same
    clones, splits and prunes."""
    rng = np.random.default_rng(70)
    n, extent = 160, 1.0
    hp = orc.AdamHyper(lr=LR, eps=1e-15)
    w0 = _params(rng, n)
    eager = [w0.copy(), np.zeros((D, n)), np.zeros((D, n)), np.zeros(n, np.uint8)]
    defer = [w0.copy(), np.zeros((D, n)), np.zeros((D, n)), np.zeros(n, np.uint8)]
    sched = _schedule(rng, n, 20)
    grads = [rng.normal(size=(D, n)) for _ in range(20)]
    _train(orc, eager, sched, grads, 0, hp, deferred=False)
    _train(orc, defer, sched, grads, 0, hp, deferred=True)
    assert defer[3].max() > 0                                  # some rows are behind
    acc, den = rng.uniform(0, 4e-4, n) * 5, np.full(n, 5.0)
    den[:7] = 0                                                # never seen: no densification
    normals = rng.normal(size=(2, 3, n))
    big = acc / 5 >= 2e-4
    n_split = int(np.sum(big[7:] & (np.exp(eager[0][3:6, 7:]).max(axis=0) > 0.01)))
    eager = list(orc.densify(*eager, 20, hp, acc, den, extent, normals[:, :, :n_split], mode=1))
    defer = list(orc.densify(*defer, 20, hp, acc, den, extent, normals[:, :, :n_split], mode=1))
    n2 = eager[0].shape[1]
    assert defer[0].shape[1] == n2 and n2 != n
    sched2 = _schedule(rng, n2, 15)
    grads2 = [rng.normal(size=(D, n2)) for _ in range(15)]
    _train(orc, eager, sched2, grads2, 20, hp, deferred=False)
    _train(orc, defer, sched2, grads2, 20, hp, deferred=True)
    wm, mm, vm = orc.adam_materialize(*defer, 35, hp, mode=1)
    np.testing.assert_array_equal(wm, eager[0])
    np.testing.assert_array_equal(mm, eager[1])
    np.testing.assert_array_equal(vm, eager[2])


def test_split_children_closed_form(orc):
    """One Gaussian rotated 90 degrees about z with scales (0.2, 0.05, 0.05):
    R maps x to y and y to -x, so the child of z = (1, 0, 0) sits at
    mu + (0, 0.2, 0) and the child of z = (0, -1, 0) at mu + (0.05, 0, 0);
    both have scales / 1.6, the parent's rotation, opacity and colour, zero
    moments and counter 0; the parent is gone."""
    hp = orc.AdamHyper(lr=LR)
    w = np.zeros((D, 2))
    w[0:3, 0] = (0.1, -0.2, 0.3)
    w[3:6, 0] = np.log([0.2, 0.05, 0.05])
    w[6:10, 0] = (math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4))
    w[10, 0] = 2.0
    w[11:14, 0] = (0.3, -0.1, 0.2)
    w[:, 1] = w[:, 0]
    w[3:6, 1] = math.log(0.001)                                # small, low gradient: untouched
    m, v = np.full((D, 2), 1e-3), np.full((D, 2), 1e-6)
    cnt = np.zeros(2, np.uint8)
    normals = np.zeros((2, 3, 1))
    normals[0, :, 0] = (1, 0, 0)
    normals[1, :, 0] = (0, -1, 0)
    W, M, V, C = orc.densify(w, m, v, cnt, 5, hp, np.array([1.0, 0.0]), np.array([1.0, 1.0]), 1.0, normals)
    assert W.shape == (D, 3)
    np.testing.assert_array_equal(W[:, 0], w[:, 1])            # the untouched Gaussian first
    np.testing.assert_allclose(W[0:3, 1], np.array([0.1, 0.0, 0.3]), atol=1e-15)
    np.testing.assert_allclose(W[0:3, 2], np.array([0.15, -0.2, 0.3]), atol=1e-15)
    for c in (1, 2):
        np.testing.assert_allclose(np.exp(W[3:6, c]), np.array([0.2, 0.05, 0.05]) / 1.6, rtol=1e-15)
        np.testing.assert_array_equal(W[6:14, c], w[6:14, 0])
        assert np.all(M[:, c] == 0) and np.all(V[:, c] == 0) and C[c] == 0
    np.testing.assert_array_equal(M[:, 0], m[:, 1])


def test_clone_catches_up_and_untouched_rows_keep_their_delay(orc):
    """A Gaussian 3 steps behind with a large gradient and small scale is
    caught up (counter 0) and cloned (the clone = its current row, zero
    moments); a Gaussian 4 steps behind that is not densified keeps its stored
    row and counter; one with opacity below 0.005 is pruned, its clone too."""
    hp = orc.AdamHyper(lr=LR, eps=1e-15)
    rng = np.random.default_rng(71)
    w = _params(rng, 3)
    w[3:6] = math.log(0.002)
    w[10] = (1.0, 1.0, -7.0)                                   # sigmoid(-7) = 0.0009
    m = rng.normal(scale=1e-3, size=(D, 3))
    v = rng.uniform(1e-8, 1e-6, size=(D, 3))
    cnt = np.array([3, 4, 0], np.uint8)
    wc, mc, vc = orc.adam_materialize(w, m, v, cnt, 30, hp, mode=1)
    acc = np.array([1.0, 0.0, 1.0])
    W, M, V, C = orc.densify(w, m, v, cnt, 30, hp, acc, np.ones(3), 1.0, np.zeros((2, 3, 0)), mode=1)
    assert W.shape == (D, 3)                                   # rows 0, 1 and the clone of 0
    np.testing.assert_array_equal(W[:, 0], wc[:, 0])
    np.testing.assert_array_equal(M[:, 0], mc[:, 0])
    np.testing.assert_array_equal(V[:, 0], vc[:, 0])
    np.testing.assert_array_equal(W[:, 1], w[:, 1])
    np.testing.assert_array_equal(M[:, 1], m[:, 1])
    np.testing.assert_array_equal(W[:, 2], wc[:, 0])
    assert np.all(M[:, 2] == 0) and np.all(V[:, 2] == 0)
    np.testing.assert_array_equal(C, [0, 4, 0])
