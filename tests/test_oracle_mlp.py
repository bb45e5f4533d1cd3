"""Pins for oracle.mlp: gradients against central finite differences and a
closed form for a single linear layer."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    dims = mlp.layer_dims(5, 7, 2, 4)
    n = sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))
    p = 0.4 * rng.standard_normal(n)
    X = rng.uniform(-1, 1, (6, 5))
    T = rng.standard_normal((6, 4))
    loss, g = mlp.loss_and_grad(p, dims, X, T)
    eps = 1e-6
    idx = rng.choice(n, size=40, replace=False)
    for i in idx:
        e = np.zeros(n)
        e[i] = eps
        lp, _ = mlp.loss_and_grad(p + e, dims, X, T)
        lm, _ = mlp.loss_and_grad(p - e, dims, X, T)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_single_linear_layer_closed_form():
    """No hidden layer: loss = |XW^T + b - T|^2 / cnt, dW = 2 (Y-T)^T X / cnt."""
    rng = np.random.default_rng(1)
    dims = mlp.layer_dims(3, 9, 0, 2)
    W = rng.standard_normal((2, 3))
    b = rng.standard_normal(2)
    p = np.concatenate([W.reshape(-1), b])
    X = rng.standard_normal((5, 3))
    T = rng.standard_normal((5, 2))
    loss, g = mlp.loss_and_grad(p, dims, X, T)
    Y = X @ W.T + b
    assert np.isclose(loss, np.mean((Y - T) ** 2))
    np.testing.assert_allclose(g[:6].reshape(2, 3), 2 * (Y - T).T @ X / Y.size)
    np.testing.assert_allclose(g[6:], 2 * (Y - T).sum(0) / Y.size)


def test_adam_first_step_is_signed_learning_rate():
    """With zero moments, the bias-corrected first step is lr * g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    z = np.zeros(50)
    p1, m1, m2 = mlp.adam_step(p, g, z, z, 1, 0.01)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(m2, 1e-3 * g * g)


def test_adam_constant_gradient_keeps_unit_step():
    """A constant gradient gives bias-corrected moments equal to g and g^2 at
    every step, so each step moves by lr * sign(g)."""
    g = np.array([3.0, -0.5, 1e-3])
    p = np.zeros(3)
    m1 = m2 = np.zeros(3)
    for step in range(1, 30):
        p_new, m1, m2 = mlp.adam_step(p, g, m1, m2, step, 0.1, eps=0.0)
        np.testing.assert_allclose(p_new - p, -0.1 * np.sign(g), rtol=1e-12)
        p = p_new
