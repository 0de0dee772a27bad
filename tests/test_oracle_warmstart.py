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
