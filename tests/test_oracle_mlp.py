"""Pins for the reference MLP: analytic gradients against central finite
differences in FP64, and Adam against its closed-form first step."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    nin, H, nout = 5, 7, 3
    rng = np.random.default_rng(1)
    theta = mlp.init(nin, H, nout, 2) + 0.01 * rng.normal(size=mlp.nparams(nin, H, nout))
    X = rng.normal(size=(11, nin))
    T = rng.normal(size=(11, nout))
    loss, g = mlp.loss_and_grad(theta, X, T, nin, H, nout)
    h = 1e-6
    num = np.zeros_like(theta)
    for k in range(len(theta)):
        e = np.zeros_like(theta)
        e[k] = h
        lp, _ = mlp.loss_and_grad(theta + e, X, T, nin, H, nout)
        lm, _ = mlp.loss_and_grad(theta - e, X, T, nin, H, nout)
        num[k] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)


def test_forward_shapes_and_relu():
    nin, H, nout = 4, 6, 2
    theta = mlp.init(nin, H, nout, 0)
    X = np.zeros((3, nin))
    y, (z1, h1, z2, h2) = mlp.forward(theta, X, nin, H, nout)
    assert y.shape == (3, nout)
    assert np.all(h1 >= 0) and np.all(h2 >= 0)
    np.testing.assert_allclose(y, 0.0)     # zero input and zero biases


def test_adam_first_step_is_signed_lr():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    t1, m, v = mlp.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, 0.01)
    # bias-corrected first step: mh = g, vh = g^2 -> update = lr * sign(g)
    np.testing.assert_allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
