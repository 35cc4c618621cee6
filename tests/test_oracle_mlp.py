"""Pins of the MLP oracle: central finite differences of the loss and the GELU
identities (no GPU)."""
import numpy as np
import pytest
from scipy.special import erf

from oracle import mlp_oracle as M


def test_gelu_identities():
    z = np.linspace(-6, 6, 241)
    # Phi(-z) = 1 - Phi(z)  =>  gelu(-z) = gelu(z) - z
    np.testing.assert_allclose(M.gelu(-z), M.gelu(z) - z, atol=1e-15)
    assert M.gelu(0.0) == 0.0
    np.testing.assert_allclose(M.gelu(np.array([8.0, 10.0])), [8.0, 10.0], atol=1e-13)
    h = 1e-6
    np.testing.assert_allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), atol=1e-9)
    assert M.gelu_grad(0.0) == pytest.approx(0.5)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    dims = M.layer_dims(6, 16, 3, 3)
    n = M.n_params(6, 16, 3, 3)
    assert n == 6 * 16 + 16 + 2 * (16 * 16 + 16) + 16 * 3 + 3
    p = rng.normal(0, 0.4, n)
    X = rng.normal(0, 1, (37, 6))
    T = rng.normal(0, 1, (37, 3))
    loss, g = M.loss_grad(p, X, T, dims)
    assert loss == pytest.approx(np.mean((M.forward(p, X, dims)[0] - T) ** 2))
    idx = rng.choice(n, 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(n)
        e[k] = h
        fd = (M.loss_grad(p + e, X, T, dims)[0] - M.loss_grad(p - e, X, T, dims)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9), k


def test_linear_network_reduces_to_least_squares_gradient():
    """One layer (no hidden activation reached): gradient of the MSE of
    X W^T + b is 2/n (Y - T)^T [X, 1]."""
    rng = np.random.default_rng(1)
    dims = [(4, 2)]
    p = rng.normal(0, 1, 4 * 2 + 2)
    X = rng.normal(0, 1, (9, 4))
    T = rng.normal(0, 1, (9, 2))
    loss, g = M.loss_grad(p, X, T, dims)
    W = p[:8].reshape(2, 4)
    b = p[8:]
    R = X @ W.T + b - T
    np.testing.assert_allclose(g[:8], (2 / R.size * R.T @ X).reshape(-1), atol=1e-14)
    np.testing.assert_allclose(g[8:], 2 / R.size * R.sum(0), atol=1e-14)
