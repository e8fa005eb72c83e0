"""The deferred update's tables (Fig. 10, §4.3.2) as the library hands them to
its kernels, against the FP64 oracle's tables.  Host-only entry point: runs on
the CPU, no device touched."""
import math

import numpy as np
import pytest

F32_REL = 2.0 ** -23     # one fp32 rounding of a double value, with margin


@pytest.fixture(scope="module")
def gs():
    from paper_2509_15645_b300 import build
    build.build()
    import paper_2509_15645_b300 as gs
    return gs


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    return oracle


def _f32(x):
    return float(np.float32(x))


@pytest.mark.parametrize("betas", [(0.9, 0.999), (0.8, 0.99)])
@pytest.mark.parametrize("max_defer", [1, 4, 15])
@pytest.mark.parametrize("t", [1, 2, 3, 9, 16, 17, 40, 1000, 1_000_000])
def test_tables_match_oracle(gs, orc, t, max_defer, betas):
    lrs = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4]
    adam = gs.adam_struct(lr=lrs, beta1=betas[0], beta2=betas[1], eps=1e-15, max_defer=max_defer)
    T = gs.adam_tables(adam, t)
    # the oracle gets the same fp32 hyper-parameters the struct carries
    b1, b2 = _f32(betas[0]), _f32(betas[1])
    hp = orc.AdamHyper(lr=[_f32(x) for x in lrs], beta1=b1, beta2=b2, eps=1e-15, max_defer=max_defer)
    for g in range(6):
        pl, ml, vl = orc.adam_lut(t, hp.lr[g], hp)
        for d in range(16):
            got = T["param"][g][d]
            if d == 0 or d > max_defer or d >= t:
                assert got == 0.0, (g, d)
            else:
                assert abs(got - pl[d]) <= F32_REL * abs(pl[d]), (g, d, got, pl[d])
                assert got > 0.0
        assert T["step_size"][g] == pytest.approx(hp.lr[g] / (1 - b1 ** t), rel=F32_REL)
    _, ml, vl = orc.adam_lut(t, hp.lr[0], hp)
    for d in range(max_defer + 1):
        assert T["mom"][d] == pytest.approx(ml[d], rel=F32_REL)
        assert T["var"][d] == pytest.approx(vl[d], rel=F32_REL)
    for d in range(16):                      # the decays are defined for every counter value
        assert T["mom"][d] == pytest.approx(b1 ** (d + 1), rel=F32_REL)
        assert T["var"][d] == pytest.approx(b2 ** (d + 1), rel=F32_REL)
    assert T["bias_corr"] == pytest.approx(math.sqrt(1 - b2 ** t), rel=F32_REL)


def test_restore_grows_with_delay(gs):
    """More skipped steps, a larger catch-up: param[g][d] increases with d, and
    scales linearly with lr (Eq. 3 is linear in lr)."""
    a1 = gs.adam_struct(lr=1e-3, max_defer=15)
    a2 = gs.adam_struct(lr=2e-3, max_defer=15)
    T1, T2 = gs.adam_tables(a1, 500), gs.adam_tables(a2, 500)
    row = T1["param"][0]
    assert all(row[d + 1] > row[d] for d in range(1, 15))
    for d in range(1, 16):
        assert T2["param"][3][d] == pytest.approx(2 * T1["param"][3][d], rel=4 * F32_REL)


@pytest.mark.parametrize("step,max_defer", [(0, 15), (-3, 15), (5, 0), (5, 16)])
def test_invalid_arguments(gs, step, max_defer):
    from paper_2509_15645_b300 import _lib
    adam = gs.adam_struct(max_defer=max_defer)
    with pytest.raises(_lib.GsError):
        gs.adam_tables(adam, step)


@pytest.mark.parametrize("wd", [0.0, 0.1, 3.0])
@pytest.mark.parametrize("t", [1, 2, 5, 16, 17, 300])
def test_adamw_tables_match_oracle(gs, orc, t, wd):
    """AdamW (decoupled decay): the restore coefficient is Fig. 10's recursion
    with its i-th term weighted by (1 - lr wd)^(i-1) and the restore's decay
    (1 - lr wd)^d, against the oracle's tables; wd = 0 gives Adam's tables."""
    from paper_2509_15645_b300 import _lib
    lrs = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4]
    adam = gs.adam_struct(lr=lrs, eps=1e-15, max_defer=15, optimizer=_lib.GS_OPT_ADAMW, weight_decay=wd)
    T = gs.adam_tables(adam, t)
    hp = orc.AdamHyper(lr=[_f32(x) for x in lrs], beta1=_f32(0.9), beta2=_f32(0.999), eps=1e-15, max_defer=15)
    A = gs.adam_tables(gs.adam_struct(lr=lrs, eps=1e-15, max_defer=15), t)
    for g in range(6):
        wl, dec = orc.adamw_lut(t, hp.lr[g], hp, _f32(wd))
        for d in range(1, 16):
            assert T["decay"][g][d] == pytest.approx(dec[d], rel=F32_REL, abs=0), (g, d)
            if d >= t:
                assert T["param"][g][d] == 0.0
            else:
                assert abs(T["param"][g][d] - wl[d]) <= F32_REL * abs(wl[d]), (g, d, T["param"][g][d], wl[d])
        if wd == 0.0:
            assert T["param"][g] == A["param"][g] and all(x == 1.0 for x in T["decay"][g])


@pytest.mark.parametrize("mu", [0.0, 0.5, 0.9])
@pytest.mark.parametrize("t", [1, 3, 40])
def test_sgdm_tables_match_oracle(gs, orc, t, mu):
    """Momentum SGD: restore coefficient lr (mu + ... + mu^d), buffer decay
    mu^(d+1), the gradient taken with weight 1, no bias correction."""
    from paper_2509_15645_b300 import _lib
    lrs = [1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3]
    adam = gs.adam_struct(lr=lrs, beta1=mu, max_defer=15, optimizer=_lib.GS_OPT_SGDM)
    T = gs.adam_tables(adam, t)
    for g in range(6):
        sl, mo = orc.sgdm_lut(_f32(lrs[g]), _f32(mu), 15)
        for d in range(1, 16):
            want = sl[d] if d < t else 0.0
            assert abs(T["param"][g][d] - want) <= F32_REL * abs(want), (g, d)
        assert T["step_size"][g] == _f32(lrs[g])
    for d in range(16):
        assert T["mom"][d] == pytest.approx(_f32(mu) ** (d + 1), rel=F32_REL, abs=1e-45)
        assert T["var"][d] == 1.0
    assert T["bias_corr"] == 1.0


@pytest.mark.parametrize("bad", [dict(optimizer=3), dict(optimizer=1, weight_decay=-0.5),
                                 dict(optimizer=1, weight_decay=float("nan")), dict(optimizer=1, weight_decay=2000.0)])
def test_invalid_optimizer_arguments(gs, bad):
    from paper_2509_15645_b300 import _lib
    with pytest.raises(_lib.GsError):
        gs.adam_tables(gs.adam_struct(lr=1e-3, **bad), 5)
