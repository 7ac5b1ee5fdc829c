"""Pins of the U-Net oracle (learned initial guess): the 3x3x3 convolution against
scipy's n-dimensional correlation, the adjoint identities of pooling and upsampling, and
the whole backward pass against central finite differences."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet


def test_conv3_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv3(x, w, b)
    for o in range(4):
        ref = b[o] + sum(ndimage.correlate(x[c], w[o, c], mode="constant", cval=0.0) for c in range(3))
        assert np.max(np.abs(y[o] - ref)) < 1e-12


def test_pool_and_up_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 6, 8))
    g = rng.standard_normal((2, 2, 3, 4))
    assert abs(np.sum(unet.pool(x) * g) - np.sum(x * unet.pool_backward(g))) < 1e-12
    assert abs(np.sum(unet.up(g) * x) - np.sum(g * unet.up_backward(x))) < 1e-12


def test_conv3_backward_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 4, 4, 4))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    gy = rng.standard_normal((3, 4, 4, 4))
    gx, gw, gb = unet.conv3_backward(x, w, gy)
    loss = lambda x_, w_, b_: float(np.sum(gy * unet.conv3(x_, w_, b_)))
    h = 1e-6
    for idx in [(0, 1, 2, 3), (1, 0, 0, 0), (1, 3, 3, 3)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert abs((loss(xp, w, b) - loss(xm, w, b)) / (2 * h) - gx[idx]) < 1e-6
    for idx in [(0, 0, 0, 0, 0), (2, 1, 1, 2, 0), (1, 1, 2, 2, 2)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        assert abs((loss(x, wp, b) - loss(x, wm, b)) / (2 * h) - gw[idx]) < 1e-6
    assert np.max(np.abs(gb - gy.sum(axis=(1, 2, 3)))) < 1e-12


@pytest.mark.parametrize("k", [0, 3, 6, 9, 10])
def test_unet_backward_finite_differences(k):
    """Whole network (crop 8, channels 2/3/4): dL/dw of several layers against central
    differences of the MSE loss."""
    rng = np.random.default_rng(4)
    params = unet.init_params(2, 3, seed=5, channels=(2, 3, 4))
    for p in params:                                # non-zero biases exercise every path
        p[1] += 0.05 * rng.standard_normal(p[1].shape)
    x = rng.standard_normal((2, 8, 8, 8))
    target = rng.standard_normal((3, 8, 8, 8))
    y, cache = unet.forward(params, x)
    _, gy = unet.mse(y, target)
    grads = unet.backward(params, cache, gy)
    h = 1e-6
    w = params[k][0]
    for flat in rng.choice(w.size, size=4, replace=False):
        idx = np.unravel_index(flat, w.shape)
        old = w[idx]
        w[idx] = old + h
        lp = unet.mse(unet.forward(params, x)[0], target)[0]
        w[idx] = old - h
        lm = unet.mse(unet.forward(params, x)[0], target)[0]
        w[idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[k][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, grads[k][0][idx])
    # bias gradient of the same layer
    bb = params[k][1]
    old = bb[0]
    bb[0] = old + h
    lp = unet.mse(unet.forward(params, x)[0], target)[0]
    bb[0] = old - h
    lm = unet.mse(unet.forward(params, x)[0], target)[0]
    bb[0] = old
    assert abs((lp - lm) / (2 * h) - grads[k][1][0]) <= 1e-6 * max(1.0, abs((lp - lm) / (2 * h)))
