"""Pins of the U-Net oracle (CPU): parameter count, layer identities, and the
analytic gradient against central finite differences (O(h^2))."""
import numpy as np
import pytest

from oracle import unet


def test_param_count():
    # 9 ci co + co per layer: 7->16, 16->16, 16->32, 32->32, 32->32, 32->32, 64->32, 32->16, 32->16, 16->3
    assert unet.num_params() == 63875


def test_conv_identity_and_shift():
    # a centre-tap identity kernel reproduces the input; an off-centre tap shifts it
    x = np.random.default_rng(0).standard_normal((2, 6, 8, 3))
    w = np.zeros((3, 3, 3, 3))
    w[1, 1] = np.eye(3)
    assert np.allclose(unet.conv3x3(x, w, np.zeros(3)), x)
    w = np.zeros((3, 3, 3, 3))
    w[1, 2] = np.eye(3)  # tap (dy=0, dx=+1): y[i, j] = x[i, j+1] with zero padding
    y = unet.conv3x3(x, w, np.zeros(3))
    assert np.allclose(y[:, :, :-1], x[:, :, 1:]) and np.all(y[:, :, -1] == 0)


def test_pool_up_adjoint():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((1, 8, 8, 2))
    b = rng.standard_normal((1, 4, 4, 2))
    # <pool(a), b> = <a, pool^T(b)> and the same for up
    assert np.isclose((unet.pool2(a) * b).sum(), (a * unet.pool2_backward(b)).sum())
    assert np.isclose((unet.up2(b) * a).sum(), (b * unet.up2_backward(a)).sum())


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    # an O(1) last layer (the default initialisation starts it near zero), so
    # that every layer's gradient is well above the round-off of the loss
    p = unet.unflatten(unet.init_params(3))
    p["d1b.w"] = p["d1b.w"] * 1e3
    theta = unet.flatten(p)
    x = rng.standard_normal((2, 8, 8, unet.CIN))
    t = rng.standard_normal((2, 8, 8, 3))
    L, g = unet.grad(theta, x, t)
    assert L == pytest.approx(unet.loss(theta, x, t), rel=1e-14)
    # one random direction per layer's weights and biases; the loss is piecewise
    # smooth (ReLU), so a step can cross a kink: take the best of three steps
    k = 0
    for name, shp in unet.param_shapes():
        m = int(np.prod(shp))
        d = np.zeros(theta.size)
        d[k:k + m] = rng.standard_normal(m)
        k += m
        errs = []
        for h in (1e-5, 1e-6, 1e-7):
            fd = (unet.loss(theta + h * d, x, t) - unet.loss(theta - h * d, x, t)) / (2 * h)
            errs.append(abs(fd - g @ d) / max(abs(g @ d), 1e-300))
        assert min(errs) < 1e-6, (name, errs)
