"""Pins of the oracle's deferred AdamW and momentum SGD (§4.3: the deferral
extends to other momentum optimizers): the eager steps against torch.optim,
the deferred ones against the eager ones through exact invariants, the AdamW
tables against their defining sum, and AdamW without decay against the
pinned Adam oracle."""
import math

import numpy as np
import pytest
import torch

GROUP_OF_ROW = [0] * 3 + [1] * 3 + [2] * 4 + [3] + [4] * 3 + [5] * 45
LR = np.array([1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3, 1e-4])


def _schedule(rng, n, steps):
    """Each step sees a window of Gaussians plus a few stragglers; 0..4 never."""
    out = []
    for _ in range(steps):
        c = rng.integers(5, n)
        lo, hi = max(5, c - n // 6), min(n, c + n // 6)
        vis = set(range(lo, hi)) | set(rng.integers(5, n, 3).tolist())
        out.append(np.array(sorted(vis), np.int32))
    return out


def _torch_params(w):
    return [torch.tensor(w[r], dtype=torch.float64, requires_grad=True) for r in range(w.shape[0])]


def test_adamw_eager_matches_torch(orc):
    rng = np.random.default_rng(10)
    D, n, wd = 14, 40, 0.05
    hp = orc.AdamHyper(lr=LR, beta1=0.9, beta2=0.999, eps=1e-8)
    w, m, v = rng.normal(size=(D, n)), np.zeros((D, n)), np.zeros((D, n))
    tw = _torch_params(w)
    opt = torch.optim.AdamW([{"params": [tw[r]], "lr": float(LR[GROUP_OF_ROW[r]])} for r in range(D)],
                            betas=(0.9, 0.999), eps=1e-8, weight_decay=wd)
    for t in range(1, 13):
        g = rng.normal(size=(D, n)) * (rng.random((D, n)) < 0.6)
        orc.adamw_eager(w, m, v, g, t, hp, wd)
        for r in range(D):
            tw[r].grad = torch.tensor(g[r], dtype=torch.float64)
        opt.step()
        np.testing.assert_allclose(w, np.stack([p.detach().numpy() for p in tw]), rtol=1e-13, atol=1e-15)


def test_sgd_momentum_eager_matches_torch(orc):
    rng = np.random.default_rng(11)
    D, n, mu = 14, 40, 0.9
    w, b = rng.normal(size=(D, n)), np.zeros((D, n))
    tw = _torch_params(w)
    opt = torch.optim.SGD([{"params": [tw[r]], "lr": float(LR[GROUP_OF_ROW[r]])} for r in range(D)], momentum=mu)
    for _ in range(12):
        g = rng.normal(size=(D, n)) * (rng.random((D, n)) < 0.6)
        orc.sgdm_eager(w, b, g, LR, mu)
        for r in range(D):
            tw[r].grad = torch.tensor(g[r], dtype=torch.float64)
        opt.step()
        np.testing.assert_allclose(w, np.stack([p.detach().numpy() for p in tw]), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("t", [2, 3, 9, 17, 300])
def test_adamw_table_recursion_equals_weighted_sum(orc, t):
    """wlut[d] = sum over the d skipped steps j = t-d..t-1 of the step's Eq. 3
    weight times rho^(t-1-j) (the decay the later skipped steps apply to it)."""
    lr, wd, b1, b2 = 2e-3, 0.1, 0.9, 0.999
    hp = orc.AdamHyper(lr=lr, beta1=b1, beta2=b2)
    wl, dec = orc.adamw_lut(t, lr, hp, wd)
    rho = 1 - lr * wd
    for d in range(0, min(15, t - 1) + 1):
        s = t - d - 1
        direct = 0.0
        for j in range(s + 1, t):
            k = j - s
            c_k = lr * b1 ** k / (1 - b1 ** j) * math.sqrt((1 - b2 ** j) / b2 ** k)
            direct += rho ** (t - 1 - j) * c_k
        assert abs(wl[d] - direct) <= 1e-13 * max(1.0, abs(direct)), (d, wl[d], direct)
        assert dec[d] == pytest.approx(rho ** d, rel=1e-15)


def _run_deferred(orc, kind, mode, steps=50, n=90, D=14, eps=1e-15, check=None, seed=12):
    rng = np.random.default_rng(seed)
    sched = _schedule(rng, n, steps)
    grads = [rng.normal(size=(D, n)) for _ in range(steps)]
    w = rng.normal(size=(D, n))
    m, v, b = np.zeros((D, n)), np.zeros((D, n)), np.zeros((D, n))
    cnt = np.zeros(n, np.uint8)
    hp = orc.AdamHyper(lr=LR, eps=eps)
    we, me, ve, be = w.copy(), m.copy(), v.copy(), b.copy()
    peak = 0
    for t, ids in enumerate(sched, start=1):
        peak = max(peak, int(cnt.max()))
        g = np.zeros((D, n))
        g[:, ids] = grads[t - 1][:, ids]
        if kind == "adamw":
            orc.adamw_deferred(w, m, v, cnt, ids, grads[t - 1][:, ids], t, hp, 0.05, mode=mode)
            orc.adamw_eager(we, me, ve, g, t, hp, 0.05)
            got = orc.adamw_materialize(w, m, v, cnt, t, hp, 0.05, mode=mode)
            check(got, (we, me, ve))
        else:
            orc.sgdm_deferred(w, b, cnt, ids, grads[t - 1][:, ids], LR, 0.9, mode=mode)
            orc.sgdm_eager(we, be, g, LR, 0.9)
            got = orc.sgdm_materialize(w, b, cnt, LR, 0.9, mode=mode)
            check(got, (we, be))
    assert peak == 15             # some Gaussians reached the counter bound (forced catch-up)


@pytest.mark.parametrize("kind", ["adamw", "sgdm"])
def test_replay_is_bit_exact_eager(orc, kind):
    def check(got, ref):
        for a, e in zip(got, ref):
            np.testing.assert_array_equal(a, e)
    _run_deferred(orc, kind, mode=1, check=check)


def test_sgd_tables_equal_eager(orc):
    """Momentum SGD's zero-gradient steps are linear and exact: the tables give
    eager SGD up to FP64 rounding at every step."""
    def check(got, ref):
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-12, atol=1e-13 * np.abs(ref[1]).max())
    _run_deferred(orc, "sgdm", mode=0, check=check)


def test_adamw_tables_exact_when_eps_is_zero(orc):
    """With eps = 0 the factorisation of each skipped step is exact, so the
    AdamW tables give eager AdamW up to FP64 rounding."""
    def check(got, ref):
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-12, atol=1e-12 * np.abs(ref[1]).max())
        np.testing.assert_allclose(got[2], ref[2], rtol=1e-12, atol=0)
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12, atol=1e-13)
    rng = np.random.default_rng(13)              # moments start positive: sqrt(v) > 0 where eps = 0
    D, n, steps = 14, 80, 45
    sched = _schedule(rng, n, steps)
    grads = [rng.normal(size=(D, n)) for _ in range(steps)]
    w = rng.normal(size=(D, n))
    m = rng.normal(scale=1e-3, size=(D, n))
    v = rng.uniform(1e-8, 1e-6, size=(D, n))
    cnt = np.zeros(n, np.uint8)
    hp = orc.AdamHyper(lr=LR, eps=0.0)
    we, me, ve = w.copy(), m.copy(), v.copy()
    for t, ids in enumerate(sched, start=1):
        g = np.zeros((D, n))
        g[:, ids] = grads[t - 1][:, ids]
        orc.adamw_deferred(w, m, v, cnt, ids, grads[t - 1][:, ids], t, hp, 0.05, mode=0)
        orc.adamw_eager(we, me, ve, g, t, hp, 0.05)
    check(orc.adamw_materialize(w, m, v, cnt, steps, hp, 0.05, mode=0), (we, me, ve))


def test_adamw_without_decay_is_adam(orc):
    """wd = 0: the AdamW tables are the Adam tables entry for entry, and the
    deferred AdamW trajectory is the (pinned) deferred Adam one — replay bit for
    bit, tables up to the order of the final step's operations."""
    for t in (2, 7, 40):
        hp = orc.AdamHyper(lr=1e-3)
        wl, dec = orc.adamw_lut(t, 1e-3, hp, 0.0)
        pl, _, _ = orc.adam_lut(t, 1e-3, hp)
        np.testing.assert_array_equal(wl, pl)
        assert np.all(dec == 1.0)
    rng = np.random.default_rng(14)
    D, n, steps = 14, 70, 40
    sched = _schedule(rng, n, steps)
    grads = [rng.normal(size=(D, n)) for _ in range(steps)]
    w0 = rng.normal(size=(D, n))
    hp = orc.AdamHyper(lr=LR, eps=1e-15)
    for mode in (1, 0):
        a = [w0.copy(), np.zeros((D, n)), np.zeros((D, n)), np.zeros(n, np.uint8)]
        b = [w0.copy(), np.zeros((D, n)), np.zeros((D, n)), np.zeros(n, np.uint8)]
        for t, ids in enumerate(sched, start=1):
            orc.adamw_deferred(*a, ids, grads[t - 1][:, ids], t, hp, 0.0, mode=mode)
            orc.adam_deferred(*b, ids, grads[t - 1][:, ids], t, hp, mode=mode)
        np.testing.assert_array_equal(a[3], b[3])
        for x, y in zip(a[:3], b[:3]):
            if mode == 1:
                np.testing.assert_array_equal(x, y)
            else:
                np.testing.assert_allclose(x, y, rtol=1e-13, atol=1e-15)
