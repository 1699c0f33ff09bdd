"""Pins of the FP64 U-Net oracle: central finite differences of the loss match
its analytic gradient, the parameter count of the 4-level network, and closed
forms of single layers."""
import numpy as np
import pytest

from oracle import unet


def test_param_count_of_the_four_level_network():
    # 3 -> 3 channels, widths (16, 32, 48, 96): about 300k parameters
    assert unet.param_count((16, 32, 48, 96)) == 299651


@pytest.mark.parametrize("widths", [(3, 5), (2, 3, 4)])
def test_gradient_matches_finite_differences(widths):
    g = np.random.default_rng(1)
    H = 8 if len(widths) == 2 else 8
    x = g.standard_normal((2, 3, H, H))
    t = g.standard_normal((2, 3, H, H))
    p = unet.init_params(widths, seed=3)
    p += 0.05 * g.standard_normal(p.size)      # biases off zero so ReLUs are not degenerate
    loss, grad = unet.loss_and_grad(p, x, t, widths)
    h = 1e-6
    idx = g.choice(p.size, size=min(60, p.size), replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (unet.loss_and_grad(p + e, x, t, widths)[0] - unet.loss_and_grad(p - e, x, t, widths)[0]) / (2 * h)
        assert fd == pytest.approx(grad[i], rel=1e-5, abs=1e-9)
    # a random direction
    v = g.standard_normal(p.size)
    fd = (unet.loss_and_grad(p + h * v, x, t, widths)[0] - unet.loss_and_grad(p - h * v, x, t, widths)[0]) / (2 * h)
    assert fd == pytest.approx(float(grad @ v), rel=1e-6)


def test_layer_closed_forms():
    g = np.random.default_rng(2)
    x = g.standard_normal((1, 2, 4, 6))
    # a centred delta kernel copies its input channel
    w = np.zeros((2, 2, 3, 3))
    w[0, 1, 1, 1] = 1.0
    w[1, 0, 1, 1] = 2.0
    y = unet.conv3(x, w, np.array([0.5, 0.0]))
    np.testing.assert_allclose(y[0, 0], x[0, 1] + 0.5)
    np.testing.assert_allclose(y[0, 1], 2 * x[0, 0])
    # a shifted delta is a cross-correlation: y[y, x] = in[y, x + 1] (zero padded)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 1, 2] = 1.0
    y = unet.conv3(x[:, :1], w, np.zeros(1))
    np.testing.assert_allclose(y[0, 0, :, :-1], x[0, 0, :, 1:])
    np.testing.assert_allclose(y[0, 0, :, -1], 0.0)
    # transposed conv with an all-ones kernel repeats each input pixel in a 2x2 block
    wt = np.ones((2, 1, 2, 2))
    y = unet.tconv(x, wt, np.zeros(1))
    np.testing.assert_allclose(y[0, 0], np.kron(x[0, 0] + x[0, 1], np.ones((2, 2))))
    np.testing.assert_allclose(unet.pool(np.kron(x, np.ones((1, 1, 2, 2)))), x)


def test_network_with_zero_weights_outputs_bias():
    widths = (4, 6)
    p = np.zeros(unet.param_count(widths))
    p[-3:] = [1.0, -2.0, 0.5]
    y = unet.forward(p, np.random.default_rng(0).standard_normal((2, 3, 8, 8)), widths)
    np.testing.assert_allclose(y[:, 0], 1.0)
    np.testing.assert_allclose(y[:, 1], -2.0)
    np.testing.assert_allclose(y[:, 2], 0.5)
