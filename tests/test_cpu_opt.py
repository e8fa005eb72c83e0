"""The host-core optimizer of the paper's offloaded configuration
(gs_cpu_deferred_step: §4.3 deferred update on the host cores;
gs_cpu_forward: §4.2.2 parameter forwarding) against the FP64 oracle's
deferred Adam, AdamW and momentum SGD.  Host arrays only: runs on the CPU."""
import numpy as np
import pytest

from helpers import hp32

U32 = 2.0 ** -23
LRS = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4]


@pytest.fixture(scope="module")
def gs():
    from paper_2509_15645_b300 import build
    build.build()
    import paper_2509_15645_b300 as gs
    return gs


def _state(n, D, seed, max_defer):
    """fp32-representable parameters and moments, counters 0..max_defer, a
    visible subset with gradients (float32 arrays; the oracle takes them as
    FP64 copies)."""
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 1.0, (D, n)).astype(np.float32)
    m = (rng.normal(0.0, 1e-3, (D, n))).astype(np.float32)
    v = (np.abs(rng.normal(0.0, 1e-6, (D, n))) + 1e-9).astype(np.float32)
    C = rng.integers(0, max_defer + 1, n).astype(np.uint8)
    vis = np.sort(rng.choice(n, n // 3, replace=False)).astype(np.int32)
    g = rng.normal(0.0, 1e-2, (D, len(vis))).astype(np.float32)
    return w, m, v, C, vis, g


def _members(C, vis, max_defer):
    """The update set of §4.3.2: visible, or the counter at its bound."""
    u = np.zeros(C.shape[0], bool)
    u[vis] = True
    u |= C == max_defer
    uids = np.nonzero(u)[0].astype(np.int32)
    return uids, C[uids].copy()


def _oracle_step(orc, kind, W, M, V, C, vis, g, t, hp, wd, mu):
    if kind == "adam":
        orc.adam_deferred(W, M, V, C, vis, g, t, hp)
    elif kind == "adamw":
        orc.adamw_deferred(W, M, V, C, vis, g, t, hp, wd)
    else:
        orc.sgdm_deferred(W, M, C, vis, g, hp.lr, mu, hp.max_defer)


def _oracle_materialize(orc, kind, W, M, V, C, t, hp, wd, mu):
    if kind == "adam":
        return orc.adam_materialize(W, M, V, C, t, hp)[0]
    if kind == "adamw":
        return orc.adamw_materialize(W, M, V, C, t, hp, wd)[0]
    return orc.sgdm_materialize(W, M, C, hp.lr, mu, hp.max_defer)[0]


def _adam(gs, kind, max_defer, wd, mu):
    if kind == "sgdm":
        return gs.adam_struct(lr=LRS, beta1=mu, eps=1e-15, max_defer=max_defer, optimizer=gs.GS_OPT_SGDM)
    return gs.adam_struct(lr=LRS, eps=1e-15, max_defer=max_defer,
                          optimizer=gs.GS_OPT_ADAMW if kind == "adamw" else gs.GS_OPT_ADAM, weight_decay=wd)


def _group_rows(D):
    """The learning-rate group of each parameter row (§2.3 layout)."""
    return [0 if r < 3 else 1 if r < 6 else 2 if r < 10 else 3 if r == 10 else 4 if r < 14 else 5 for r in range(D)]


@pytest.mark.parametrize("kind", ["adam", "adamw", "sgdm"])
@pytest.mark.parametrize("plane0", [0, 11])
def test_cpu_deferred_step_matches_oracle(gs, orc, kind, plane0):
    n, D, t, max_defer, wd, mu = 6000, 23, 20, 15, 0.05, 0.9
    w, m, v, C, vis, g = _state(n, D, 11 + plane0, max_defer)
    if kind == "sgdm":
        v[:] = 0.0
    hp = hp32(orc, lr=LRS, beta1=mu if kind == "sgdm" else 0.9, max_defer=max_defer)
    W, M, V, Cc = w.astype(np.float64), m.astype(np.float64), v.astype(np.float64), C.copy()
    _oracle_step(orc, kind, W, M, V, Cc, vis, g.astype(np.float64), t, hp, wd, mu)
    uids, udelay = _members(C, vis, max_defer)
    adam = _adam(gs, kind, max_defer, wd, mu)
    rows = slice(plane0, D)
    w2, m2, v2, g2 = (np.ascontiguousarray(a[rows].T) for a in (w, m, v, g))     # one row per Gaussian
    gs.cpu_deferred_step(w2, m2, v2, plane0, uids, udelay, vis, g2, adam, t, threads=4)
    w2, m2, v2 = w2.T, m2.T, v2.T
    grp = np.asarray(_group_rows(D))[rows]
    lr = np.asarray(LRS)[grp]
    d = C.astype(np.float64)
    dirmag = (np.abs(m[rows]) + 1e-2) if kind == "sgdm" else (np.abs(m[rows]) + 1e-2) / np.sqrt(v[rows] + 1e-12)
    bw = 16 * U32 * np.abs(W[rows]) + 64 * U32 * lr[:, None] * (d[None, :] + 2) * dirmag
    assert np.all(np.abs(w2 - W[rows]) <= bw), float(np.max(np.abs(w2 - W[rows]) / bw))
    bm = 8 * U32 * (np.abs(m[rows]) + np.abs(M[rows])) + 1e-30
    assert np.all(np.abs(m2 - M[rows]) <= bm), float(np.max(np.abs(m2 - M[rows]) / bm))
    if kind != "sgdm":
        bv = 8 * U32 * (np.abs(v[rows]) + np.abs(V[rows])) + 1e-30
        assert np.all(np.abs(v2 - V[rows]) <= bv), float(np.max(np.abs(v2 - V[rows]) / bv))
    # non-members are untouched bit for bit
    keep = np.ones(n, bool)
    keep[uids] = False
    np.testing.assert_array_equal(w2[:, keep], w[rows][:, keep])
    np.testing.assert_array_equal(m2[:, keep], m[rows][:, keep])


@pytest.mark.parametrize("kind", ["adam", "adamw", "sgdm"])
def test_cpu_forward_is_the_next_steps_view(gs, orc, kind):
    """Forwarding from the stored state plus the pending update of step t gives
    what the oracle's state after step t restores for step t + 1 (members of
    the update: their new values; the others: the deferred restore), and leaves
    the host arrays as they were."""
    n, D, t, max_defer, wd, mu = 6000, 23, 20, 15, 0.05, 0.9
    w, m, v, C, vis, g = _state(n, D, 21, max_defer)
    if kind == "sgdm":
        v[:] = 0.0
    hp = hp32(orc, lr=LRS, beta1=mu if kind == "sgdm" else 0.9, max_defer=max_defer)
    W, M, V, C1 = w.astype(np.float64), m.astype(np.float64), v.astype(np.float64), C.copy()
    _oracle_step(orc, kind, W, M, V, C1, vis, g.astype(np.float64), t, hp, wd, mu)
    want = _oracle_materialize(orc, kind, W, M, V, C1, t, hp, wd, mu)
    uids, udelay = _members(C, vis, max_defer)
    ids = np.sort(np.random.default_rng(5).choice(n, n // 2, replace=False)).astype(np.int32)
    adam = _adam(gs, kind, max_defer, wd, mu)
    wr, mr, vr, gr = (np.ascontiguousarray(a.T) for a in (w, m, v, g))     # one row per Gaussian
    out = gs.cpu_forward(wr, mr, vr, 0, ids, C1[ids], uids, udelay, vis, gr, adam, t, threads=3)
    np.testing.assert_array_equal(wr, w.T)
    np.testing.assert_array_equal(mr, m.T)
    np.testing.assert_array_equal(vr, v.T)
    assert (C1[ids] == 0).sum() > 100 and (C1[ids] > 0).sum() > 100
    grp = np.asarray(_group_rows(D))
    lr = np.asarray(LRS)[grp]
    d = np.maximum(C[ids], C1[ids]).astype(np.float64)
    mm, vv = m[:, ids], v[:, ids]
    dirmag = (np.abs(mm) + 1e-2) if kind == "sgdm" else (np.abs(mm) + 1e-2) / np.sqrt(vv + 1e-12)
    b = 16 * U32 * np.abs(want[:, ids]) + 64 * U32 * lr[:, None] * (d[None, :] + 2) * dirmag
    err = np.abs(out - want[:, ids])
    assert np.all(err <= b), float(np.max(err / b))
    # nothing pending: counter 0 takes the stored value as it is
    out0 = gs.cpu_forward(wr, mr, vr, 0, ids, np.zeros(len(ids), np.uint8), np.zeros(0, np.int32),
                          np.zeros(0, np.uint8), np.zeros(0, np.int32), np.zeros((0, D), np.float32), adam, t)
    np.testing.assert_array_equal(out0, w[:, ids])


def test_cpu_optimizer_rejects_bad_arguments(gs):
    from paper_2509_15645_b300 import _lib
    n, D = 100, 23
    w, m, v, C, vis, g = (np.ascontiguousarray(a.T) if a.ndim == 2 else a for a in _state(n, D, 3, 15))
    adam = gs.adam_struct(lr=LRS)
    uids = np.array([5, 3], np.int32)                   # not ascending
    with pytest.raises(_lib.GsError):
        gs.cpu_deferred_step(w, m, v, 0, uids, np.zeros(2, np.uint8), vis, g, adam, 3)
    with pytest.raises(_lib.GsError):                   # delay above max_defer
        gs.cpu_deferred_step(w, m, v, 0, np.array([1], np.int32), np.array([16], np.uint8), vis, g, adam, 3)
    with pytest.raises(_lib.GsError):                   # rows beyond the parameter vector
        gs.cpu_deferred_step(w, m, v, 40, np.array([1], np.int32), np.zeros(1, np.uint8), vis, g, adam, 3)
    with pytest.raises(_lib.GsError):                   # step 0 has nothing to apply
        gs.cpu_deferred_step(w, m, v, 0, np.array([1], np.int32), np.zeros(1, np.uint8), vis, g, adam, 0)
    eager = gs.adam_struct(lr=LRS, mode=_lib.GS_ADAM_EAGER)
    with pytest.raises(_lib.GsError):
        gs.cpu_deferred_step(w, m, v, 0, np.array([1], np.int32), np.zeros(1, np.uint8), vis, g, eager, 3)
