"""Pins of the oracle's optimizer: eager Adam (Eq. 1) against torch.optim.Adam
and a closed form; deferred Adam (Eqs. 2-3, Fig. 10, §4.3.2) against eager
Adam through exact invariants; the paper's printed constants."""
import json
import math
import os

import numpy as np
import pytest
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
GROUP_OF_ROW = [0] * 3 + [1] * 3 + [2] * 4 + [3] + [4] * 3 + [5] * 45


def _state(rng, D, n, positive_moments=True):
    w = rng.normal(size=(D, n))
    m = rng.normal(scale=1e-3, size=(D, n)) if positive_moments else np.zeros((D, n))
    v = rng.uniform(1e-8, 1e-6, size=(D, n)) if positive_moments else np.zeros((D, n))
    return w, m, v


def test_eager_matches_torch_adam(orc):
    rng = np.random.default_rng(0)
    D, n = 14, 50
    lr = np.array([1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3, 1e-4])
    hp = orc.AdamHyper(lr=lr, beta1=0.9, beta2=0.999, eps=1e-8)
    w, m, v = _state(rng, D, n, positive_moments=False)
    tw = [torch.tensor(w[r], dtype=torch.float64, requires_grad=True) for r in range(D)]
    opt = torch.optim.Adam([{"params": [tw[r]], "lr": float(lr[GROUP_OF_ROW[r]])} for r in range(D)],
                           betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 13):
        g = rng.normal(size=(D, n)) * (rng.random((D, n)) < 0.6)
        orc.adam_eager(w, m, v, g, t, hp)
        for r in range(D):
            tw[r].grad = torch.tensor(g[r], dtype=torch.float64)
        opt.step()
        got = np.stack([p.detach().numpy() for p in tw])
        np.testing.assert_allclose(w, got, rtol=1e-13, atol=1e-15)


def test_eager_constant_gradient_closed_form(orc):
    """Constant g: m_hat = g and v_hat = g^2 exactly, so each step moves w by
    lr g / (|g| + eps)."""
    rng = np.random.default_rng(1)
    D, n, steps = 14, 20, 40
    hp = orc.AdamHyper(lr=1e-3, eps=1e-15)
    w, m, v = _state(rng, D, n, positive_moments=False)
    g = rng.normal(size=(D, n))
    w0 = w.copy()
    for t in range(1, steps + 1):
        orc.adam_eager(w, m, v, g, t, hp)
    np.testing.assert_allclose(w, w0 - steps * 1e-3 * g / (np.abs(g) + 1e-15), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("t", [2, 3, 9, 17, 40, 1000])
def test_lut_recursion_equals_eq3_sum(orc, t):
    """param_lut[d] built by the recursion of Fig. 10 equals the w_scale sum of
    Eq. 3 written out term by term."""
    hp = orc.AdamHyper(lr=1e-3, beta1=0.9, beta2=0.999)
    pl, ml, vl = orc.adam_lut(t, 1e-3, hp)
    b1, b2 = 0.9, 0.999
    for d in range(0, min(15, t - 1) + 1):
        direct = sum(1e-3 / math.sqrt(b2 ** (l + 1) / (1 - b2 ** (t - d + l))) * b1 ** (l + 1) /
                     (1 - b1 ** (t - d + l)) for l in range(d))
        assert abs(pl[d] - direct) <= 1e-13 * max(1.0, abs(direct))
        assert ml[d] == pytest.approx(b1 ** (d + 1), rel=1e-15)
        assert vl[d] == pytest.approx(b2 ** (d + 1), rel=1e-15)
    assert np.all(np.isnan(pl[t:])) if t <= 15 else True


def _visibility_schedule(rng, n, steps):
    """Each step sees a contiguous window of Gaussians plus a few stragglers;
    Gaussians 0..4 are never seen."""
    out = []
    for _ in range(steps):
        c = rng.integers(5, n)
        lo, hi = max(5, c - n // 6), min(n, c + n // 6)
        vis = set(range(lo, hi)) | set(rng.integers(5, n, 3).tolist())
        out.append(np.array(sorted(vis), np.int32))
    return out


def _run(orc, w, m, v, cnt, sched, grads, hp, mode, geo_eager=False, materialize_each=None):
    for t, ids in enumerate(sched, start=1):
        orc.adam_deferred(w, m, v, cnt, ids, grads[t - 1][:, ids], t, hp, mode=mode, geo_eager=geo_eager)
        if materialize_each is not None:
            materialize_each(t, w, m, v, cnt)


def test_deferred_replay_is_bit_exact_eager(orc):
    """Replaying the skipped zero-gradient steps through Eq. 1 reproduces eager
    Adam bit for bit (same operations in the same order)."""
    rng = np.random.default_rng(2)
    D, n, steps = 14, 120, 60
    hp = orc.AdamHyper(lr=np.array([1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3, 1e-4]), eps=1e-15)
    sched = _visibility_schedule(rng, n, steps)
    grads = [rng.normal(size=(D, n)) for _ in range(steps)]
    w, m, v = _state(rng, D, n, positive_moments=False)
    we, me, ve = w.copy(), m.copy(), v.copy()
    cnt = np.zeros(n, np.uint8)

    def check(t, w_, m_, v_, c_):
        g = np.zeros((D, n))
        g[:, sched[t - 1]] = grads[t - 1][:, sched[t - 1]]
        orc.adam_eager(we, me, ve, g, t, hp)
        wm, mm, vm = orc.adam_materialize(w_, m_, v_, c_, t, hp, mode=1)
        np.testing.assert_array_equal(wm, we)
        np.testing.assert_array_equal(mm, me)
        np.testing.assert_array_equal(vm, ve)

    _run(orc, w, m, v, cnt, sched, grads, hp, mode=1, materialize_each=check)


def test_deferred_lut_exact_when_eps_is_zero(orc):
    """With eps = 0 the factorisation of Eq. 3 is exact, so the table form
    equals eager Adam up to FP64 rounding; only eps separates them."""
    rng = np.random.default_rng(3)
    D, n, steps = 14, 100, 50
    hp = orc.AdamHyper(lr=1e-3, eps=0.0)
    sched = _visibility_schedule(rng, n, steps)
    grads = [rng.normal(size=(D, n)) for _ in range(steps)]
    w, m, v = _state(rng, D, n)                 # mid-training state: v > 0 everywhere
    we, me, ve = w.copy(), m.copy(), v.copy()
    cnt = np.zeros(n, np.uint8)
    _run(orc, w, m, v, cnt, sched, grads, hp, mode=0)
    for t in range(1, steps + 1):
        g = np.zeros((D, n))
        g[:, sched[t - 1]] = grads[t - 1][:, sched[t - 1]]
        orc.adam_eager(we, me, ve, g, t, hp)
    wm, mm, vm = orc.adam_materialize(w, m, v, cnt, steps, hp, mode=0)
    # m is a sum of terms of both signs: allow rounding relative to its scale
    np.testing.assert_allclose(mm, me, rtol=1e-12, atol=1e-12 * np.abs(me).max())
    np.testing.assert_allclose(vm, ve, rtol=1e-12, atol=0)
    np.testing.assert_allclose(wm, we, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("eps", [1e-15, 1e-8, 1e-6])
def test_deferred_lut_eps_error_bound(orc, eps):
    """One catch-up of d deferred steps: |w_table - w_exact| is bounded by the
    sum over the skipped steps of the eps-factoring error of Eq. 3,
    X eps |a - 1| / ((a sqrt(v) + eps) a (sqrt(v) + eps)),
    with X = lr b1^(l+1) m / (1 - b1^s) and a = sqrt(b2^(l+1) / (1 - b2^s))."""
    rng = np.random.default_rng(4)
    D, n = 14, 64
    b1, b2, lr = 0.9, 0.999, 1e-3
    hp = orc.AdamHyper(lr=lr, eps=eps)
    t0 = 7
    for d in [1, 5, 15]:
        w, m, v = _state(rng, D, n)
        cnt = np.full(n, d, np.uint8)
        ids = np.arange(0, n, 2, dtype=np.int32)
        gc = rng.normal(size=(D, ids.size))
        wl, ml_, vl_ = w.copy(), m.copy(), v.copy()
        wr, mr, vr = w.copy(), m.copy(), v.copy()
        t = t0 + d
        orc.adam_deferred(wl, ml_, vl_, cnt.copy(), ids, gc, t, hp, mode=0)
        orc.adam_deferred(wr, mr, vr, cnt.copy(), ids, gc, t, hp, mode=1)
        bound = np.zeros((D, n))
        for l in range(d):
            s = t - d + l
            X = lr * b1 ** (l + 1) * np.abs(m) / (1 - b1 ** s)
            a = math.sqrt(b2 ** (l + 1) / (1 - b2 ** s))
            bound += X * eps * abs(a - 1) / ((a * np.sqrt(v) + eps) * a * (np.sqrt(v) + eps))
        # the step at t then amplifies nothing: it uses the same m_new / v_new on both sides
        slack = 64 * np.finfo(np.float64).eps * (np.abs(w) + lr * (d + 1))
        assert np.all(np.abs(wl - wr) <= bound + slack)
        if eps >= 1e-6:
            assert np.max(np.abs(wl - wr)) > 10 * np.max(slack)   # the approximation is really there
        np.testing.assert_allclose(ml_, mr, rtol=1e-13)
        np.testing.assert_allclose(vl_, vr, rtol=1e-13)


def test_counter_period_and_wasted_updates(orc):
    """A Gaussian that is never seen is caught up exactly when its counter
    reaches MAX = 15: every 16th step, i.e. 1/16 of the steps (<= the paper's
    1/15 = 6.7% bound)."""
    D, n, steps = 14, 8, 64
    hp = orc.AdamHyper()
    w, m, v = _state(np.random.default_rng(5), D, n)
    cnt = np.zeros(n, np.uint8)
    seen = np.array([3], np.int32)
    history = []
    for t in range(1, steps + 1):
        orc.adam_deferred(w, m, v, cnt, seen, np.ones((D, 1)), t, hp)
        history.append(cnt.copy())
    h = np.array(history)
    assert np.all(h[:, 3] == 0)
    np.testing.assert_array_equal(h[:, 0], np.arange(1, steps + 1) % 16)
    updates = np.count_nonzero(h[:, 0] == 0)
    assert updates == steps // 16
    assert updates / steps <= 1 / 15


def test_geometry_eager_mode(orc):
    """geo_eager: mean/scale/quaternion rows follow eager Adam bit for bit; the
    remaining rows are deferred."""
    rng = np.random.default_rng(6)
    D, n, steps = 14, 60, 30
    hp = orc.AdamHyper(eps=1e-15)
    sched = _visibility_schedule(rng, n, steps)
    grads = [rng.normal(size=(D, n)) for _ in range(steps)]
    w, m, v = _state(rng, D, n, positive_moments=False)
    we, me, ve = w.copy(), m.copy(), v.copy()
    cnt = np.zeros(n, np.uint8)
    _run(orc, w, m, v, cnt, sched, grads, hp, mode=1, geo_eager=True)
    for t in range(1, steps + 1):
        g = np.zeros((D, n))
        g[:, sched[t - 1]] = grads[t - 1][:, sched[t - 1]]
        orc.adam_eager(we, me, ve, g, t, hp)
    np.testing.assert_array_equal(w[:10], we[:10])
    wm, mm, vm = orc.adam_materialize(w, m, v, cnt, steps, hp, mode=1, geo_eager=True)
    np.testing.assert_array_equal(wm, we)


def test_paper_printed_constants(orc):
    """Constants the paper prints (tests/golden/paper_constants.json)."""
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as f:
        c = json.load(f)
    assert orc.n_params(3) == c["params_per_gaussian"]
    assert round(c["geometric_params"] / c["params_per_gaussian"], 2) == c["geometric_memory_fraction"]
    assert c["max_counter"] < 2 ** c["counter_bits"]
    assert round(1 / c["max_counter"], 3) == c["wasted_update_bound"]
    # a full Adam step touches 4D reads + 3D writes of 32-bit words
    assert 4 + 3 == c["adam_words_per_param"]
    assert 7 * 59 * 4 == 1652
