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


def test_bf16_round_is_round_to_nearest_even():
    """bf16_round against exact cases of the definition (8 significand bits, ties to even)
    and against torch's float32 -> bfloat16 conversion on values over 17 decades."""
    from oracle.unet import bf16_round
    one = 1.0
    cases = {one: one, one + 2.0 ** -8: one, one + 3 * 2.0 ** -8: one + 2.0 ** -6,
             one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7, -3.0: -3.0, 2.0 ** -130: 2.0 ** -130}
    for a, b in cases.items():
        assert bf16_round(np.array([a]))[0] == b, (a, b)
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bf16_round(a), ref)


def test_bf16_storage_form_without_rounding_is_the_network():
    """store = identity reproduces the plain forward and backward exactly."""
    from oracle import unet as ou
    params = ou.init_params(2, 2, seed=1, channels=(2, 3, 4))
    x = np.random.default_rng(2).standard_normal((2, 4, 4, 4))
    y0, c0 = ou.forward(params, x)
    y1, c1 = ou.forward(params, x, store=lambda a: a)
    assert np.array_equal(y0, y1)
    g0 = ou.backward(params, c0, y0)
    g1 = ou.backward(params, c1, y1, store=lambda a: a)
    assert all(np.array_equal(a, b) for p, q in zip(g0, g1) for a, b in zip(p, q))
