"""Pins for the oracle's Newton-guess network: gradient vs central finite
differences (FP64), GELU vs its integral definition, shapes."""
import numpy as np
from scipy import integrate

from oracle.mlp import N_PARAMS, forward, gelu, gelu_prime, loss_and_grad


def test_parameter_count():
    assert N_PARAMS == 4609


def test_gelu_is_x_times_normal_cdf():
    for x in (-3.0, -0.7, 0.0, 0.4, 2.5):
        cdf, _ = integrate.quad(lambda u: np.exp(-0.5 * u * u) / np.sqrt(2 * np.pi), -np.inf, x)
        assert abs(gelu(np.array([x]))[0] - x * cdf) < 1e-13
        h = 1e-5
        fd = (gelu(np.array([x + h]))[0] - gelu(np.array([x - h]))[0]) / (2 * h)
        assert abs(gelu_prime(np.array([x]))[0] - fd) < 1e-9


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, N_PARAMS)
    X = rng.normal(0, 1, (40, 5))
    t = rng.normal(0, 1, 40)
    _, g = loss_and_grad(theta, X, t)
    idx = rng.choice(N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [N_PARAMS - 1, 0, 320, 384, 4480]])
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (loss_and_grad(tp, X, t)[0] - loss_and_grad(tm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])
    y, _ = forward(theta, X)
    assert y.shape == (40,)
