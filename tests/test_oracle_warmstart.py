"""Pins for the warm-start reference (no GPU): the conv against scipy's
correlate, every gradient against central finite differences."""

import numpy as np
import pytest

from oracle import warmstart as ows


def test_conv3d_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 4, 6, 3))
    W = rng.standard_normal((3, 3, 3, 3, 2))
    b = rng.standard_normal(2)
    y = ows.conv3d(x, W, b)
    for o in range(2):
        ref = b[o] + sum(ndimage.correlate(x[..., i], W[..., i, o], mode="constant", cval=0.0) for i in range(3))
        assert np.abs(y[..., o] - ref).max() < 1e-12


def test_conv3d_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 3, 2))
    W = rng.standard_normal((3, 3, 3, 2, 3))
    dy = rng.standard_normal((3, 4, 3, 3))
    dx, dW, db = ows.conv3d_backward(x, W, dy)
    h = 1e-6
    f = lambda x_, W_: (dy * ows.conv3d(x_, W_)).sum()
    for idx in [(0, 0, 0, 0), (2, 3, 2, 1), (1, 2, 1, 0)]:
        e = np.zeros_like(x); e[idx] = h
        assert abs((f(x + e, W) - f(x - e, W)) / (2 * h) - dx[idx]) < 1e-6
    for idx in [(0, 0, 0, 0, 0), (2, 1, 0, 1, 2), (1, 1, 1, 0, 1)]:
        e = np.zeros_like(W); e[idx] = h
        assert abs((f(x, W + e) - f(x, W - e)) / (2 * h) - dW[idx]) < 1e-6
    assert np.allclose(db, dy.sum(axis=(0, 1, 2)))


def test_network_gradients_finite_differences():
    rng = np.random.default_rng(2)
    shape = (3, 4, 4)
    x = rng.standard_normal(shape + (8,))
    params = [(0.3 * rng.standard_normal((3, 3, 3, ci, co)), 0.1 * rng.standard_normal(co))
              for ci, co in [(8, 6), (6, 6), (6, 6), (6, 4)]]
    target = rng.standard_normal(shape + (2,))
    support = (rng.random(shape + (2,)) > 0.5).astype(float)
    support[0, 0, 0, 1] = -1.0                      # a ghost coordinate
    def L(ps):
        y, _ = ows.forward(x, ps)
        return ows.loss_and_grad(y, target, support)[0]
    y, acts = ows.forward(x, params)
    loss, dy = ows.loss_and_grad(y, target, support)
    grads = ows.backward(acts, params, dy)
    h = 1e-6
    for li, widx in [(0, (1, 1, 1, 3, 2)), (1, (0, 2, 1, 5, 0)), (3, (2, 0, 1, 4, 3))]:
        W, b = params[li]
        Wp, Wm = W.copy(), W.copy()
        Wp[widx] += h
        Wm[widx] -= h
        pp = list(params); pp[li] = (Wp, b)
        pm = list(params); pm[li] = (Wm, b)
        fd = (L(pp) - L(pm)) / (2 * h)
        assert abs(fd - grads[li][0][widx]) < 1e-6 * max(1, abs(fd))
    b = params[2][1]
    bp, bm = b.copy(), b.copy()
    bp[1] += h
    bm[1] -= h
    pp = list(params); pp[2] = (params[2][0], bp)
    pm = list(params); pm[2] = (params[2][0], bm)
    assert abs((L(pp) - L(pm)) / (2 * h) - grads[2][1][1]) < 1e-6


GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(__import__("os").path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_features_and_targets_golden():
    """Hand-derived features and targets on the 4 x 3 x 3 slot grid of a 3 x 3 x 6 grid
    (a wrong frequency coordinate, slot order or soft threshold fails here)."""
    rows = _golden_lines("ws_features_3x3x6.txt")
    lam = float(rows[0][1])
    dims = (3, 3, 6)
    c = np.zeros((4, 3, 3, 2))
    slots = []
    for r in rows:
        if r[0] == "SLOT":
            kl, k1, k2 = (int(v) for v in r[1:4])
            c[kl, k1, k2] = [float(r[5]), float(r[6])]
            slots.append(((kl, k1, k2), [float(v) for v in r[8:16]]))
    x = ows.features(c.reshape(-1), lam, dims)
    assert x.shape == (4, 3, 3, 8)
    for idx, ref in slots:
        assert np.allclose(x[idx], ref, rtol=0, atol=1e-15), (idx, x[idx], ref)
    # the slots with c = 0: only the frequency coordinates are non-zero
    third = [0.0, 2 / 3, 2 / 3]
    for kl in range(4):
        for k1 in range(3):
            for k2 in range(3):
                if any(idx == (kl, k1, k2) for idx, _ in slots):
                    continue
                assert np.allclose(x[kl, k1, k2], [0, 0, 0, 0, 0, kl / 3, third[k1], third[k2]], atol=1e-15)
    b = np.zeros((4, 3, 3, 2))
    ghost = np.zeros((4, 3, 3, 2), dtype=bool)
    targets = []
    for r in rows:
        if r[0] == "TARGET":
            idx = tuple(int(v) for v in r[1:4])
            b[idx] = [float(r[5]), float(r[6])]
            targets.append((idx, [float(r[8]), float(r[9])], [float(r[11]), float(r[12])]))
        elif r[0] == "GHOST":
            ghost[tuple(int(v) for v in r[1:5])] = True
    t, sup = ows.targets(c.reshape(-1), b.reshape(-1), lam, dims, ghost.reshape(-1))
    for idx, tref, sref in targets:
        assert np.allclose(t[idx], tref, atol=1e-15) and np.array_equal(sup[idx], sref)
    assert sup[0, 0, 0, 1] == -1 and sup[0, 0, 0, 0] == 0


def test_start_point_golden_and_invariants():
    """Hand-derived start points, and what the construction guarantees at any input:
    s1 nu1 = s2 nu2 = mu0, z - beta - s2 = z + beta - s1 = 0, s > 0, nu > 0."""
    rows = _golden_lines("ws_start_point.txt")
    lam, mu_scale = float(rows[0][1]), float(rows[1][1])
    for r in rows[2:]:
        c, y, lg = (float(v) for v in r[1:4])
        ref = [float(v) for v in r[5:11]]
        got = [float(v) for v in ows.start_point(c, y, lg, lam, mu_scale)]
        assert np.allclose(got, ref, rtol=1e-15, atol=1e-15), (got, ref)
    rng = np.random.default_rng(3)
    c, y, lg = 3 * rng.standard_normal(1000), rng.standard_normal(1000), 4 * rng.standard_normal(1000)
    beta, z, s1, s2, nu1, nu2 = ows.start_point(c, y, lg, 0.7, 0.3)
    mu0 = 0.3 * 0.7 ** 2
    assert np.all(s1 > 0) and np.all(s2 > 0) and np.all(nu1 > 0) and np.all(nu2 > 0)
    assert np.allclose(s1 * nu1, mu0, rtol=1e-14) and np.allclose(s2 * nu2, mu0, rtol=1e-14)
    assert np.allclose(z + beta - s1, 0, atol=1e-14) and np.allclose(z - beta - s2, 0, atol=1e-14)
