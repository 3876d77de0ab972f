"""Pins of the FP64 reference network used to check the device training
kernels: the analytic gradient equals central finite differences of the loss,
and a plain gradient-descent loop on it reduces the loss of a smooth map."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(60)
    theta = mlp.init(1) + 0.05 * rng.normal(size=mlp.N_PARAMS)
    x = rng.uniform(-1, 1, (32, 3))
    p = rng.uniform(0, 1, (32, 3))
    L, g = mlp.loss_grad(theta, x, p)
    assert L == mlp.loss(theta, x, p)
    idx = rng.choice(mlp.N_PARAMS, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss(theta + e, x, p) - mlp.loss(theta - e, x, p)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(g[i]), (i, fd, g[i])


def test_descent_reduces_loss_on_smooth_map():
    rng = np.random.default_rng(61)
    theta = mlp.init(2)
    x = rng.uniform(-1, 1, (512, 3))
    p = 0.5 + 0.4 * np.tanh(x @ np.array([[0.7, 0.2, 0.0], [0.1, 0.8, 0.1], [0.0, 0.3, 0.6]]))
    L0 = mlp.loss(theta, x, p)
    for _ in range(300):
        L, g = mlp.loss_grad(theta, x, p)
        theta -= 0.05 * g
    assert mlp.loss(theta, x, p) < 0.2 * L0
