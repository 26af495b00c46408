"""Pins of the network reference: the convolution against scipy.ndimage.correlate, the
backward pass against central finite differences, and the identity kernel."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import convnet


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 5, 6, 7))
    W = rng.normal(size=(2, 3, 3, 3, 3))
    b = rng.normal(size=2)
    y = convnet.conv(x, W, b)
    for o in range(2):
        ref = b[o] + sum(ndimage.correlate(x[c], W[o, c], mode="constant", cval=0.0) for c in range(3))
        np.testing.assert_allclose(y[o], ref, rtol=1e-12, atol=1e-12)


def test_identity_kernel():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 4, 4, 4))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 1, 1, 1] = 1.0
    np.testing.assert_array_equal(convnet.conv(x, W), x)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = convnet.init_params(rng, (3, 4, 4, 4, 1))
    params = [(W, rng.normal(scale=0.1, size=b.shape)) for W, b in params]
    x = rng.normal(size=(3, 4, 5, 6))
    t = rng.normal(size=(1, 4, 5, 6))
    mask = np.ones_like(t)
    mask[:, 0] = 0.0

    def loss_of(ps, xx):
        y, _ = convnet.forward(ps, xx)
        return convnet.mse(y, t, mask)[0]

    y, cache = convnet.forward(params, x)
    _, dy = convnet.mse(y, t, mask)
    grads, gx = convnet.backward(params, cache, dy)
    h = 1e-6
    for li in range(4):
        W, b = params[li]
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in W.shape)
            Wp = W.copy(); Wp[idx] += h
            Wm = W.copy(); Wm[idx] -= h
            pp = list(params); pp[li] = (Wp, b)
            pm = list(params); pm[li] = (Wm, b)
            fd = (loss_of(pp, x) - loss_of(pm, x)) / (2 * h)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8)
        o = rng.integers(0, b.shape[0])
        bp = b.copy(); bp[o] += h
        bm = b.copy(); bm[o] -= h
        pp = list(params); pp[li] = (W, bp)
        pm = list(params); pm[li] = (W, bm)
        fd = (loss_of(pp, x) - loss_of(pm, x)) / (2 * h)
        assert grads[li][1][o] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        fd = (loss_of(params, xp) - loss_of(params, xm)) / (2 * h)
        assert gx[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8)
